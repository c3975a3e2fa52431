"""Benchmark of the SMC hot path: particle-updates/s per SMC iteration.

Workload (one "step" = one full SMC iteration over all particles): the
almost-constant-velocity particle filter of Sec. 5.1 at N = 2^20 particles,
FP32 per particle with FP64 normaliser and evidence, 1000 synthetic
observations (seed 0), ESS threshold 0.5 N; move + weight + normaliser + ESS
test + (when due) fixed-point CDF and ancestor selection; the gather runs in
the next move.  The headline scheme is systematic; the other three schemes
are reported under "per_scheme".

Timing: W untimed warm-up iterations, then K timed iterations.  Before each
timed iteration a 1 GB buffer is written (8x the 126 MB L2), outside the
timed events; every iteration is bracketed by CUDA events on the stream
the kernels run on.  Under torchrun each rank runs an independent replica
(another seed); the max over ranks of the timed region is used.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (a few iterations at the full N) on the host cores.
"""
import argparse
import ctypes
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FULL = 1 << 20
T_OBS = 1000
METRIC = "particle-updates/s per SMC iteration at N=2^20"
WORKLOAD = "cv-pf N=2^20 T=1000 fp32 (fp64 normaliser) ESS<0.5N"
# algorithmic HBM bytes per particle of the fused move/weight kernel:
# state read 16 B (gathered after a resampling step) + state write 16 B +
# log-weight write 4 B + log-weight read 4 B (or the ancestor index read 4 B
# after a resampling step)
PF_BYTES_PER_PARTICLE = 40
SCAN_BYTES_PER_PARTICLE = 12     # log-weight read 4 B + CDF write 8 B
SELECT_BYTES_PER_PARTICLE = 12   # CDF read 8 B + ancestor write 4 B
FLUSH_BYTES = 1 << 30  # written between timed iterations: 8x the 126 MB L2
HEAD_START = 8         # extra flushes queued before the timed loop so the host runs ahead of the GPU
# kernels of one resampling step (one cooperative kernel for every scheme,
# launched every iteration; it exits after reading the state block when the
# ESS test did not ask for resampling)
RESAMPLE_KERNELS = {"systematic": 1, "stratified": 1, "multinomial": 1, "residual": 1,
                    "residual_systematic": 1, "residual_stratified": 1}
# algorithmic bytes per particle of a resampling step beyond the move:
# log-weight re-read 4 B + ancestor write 4 B + ancestor read 4 B
RESAMPLE_BYTES_PER_PARTICLE = 12
# DRAM bytes (read + write) of one launch of the move kernel, from the ncu
# capture summarised in this file (null when the file is absent)
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "pf_iterate_cv_gather_2e20.md")


def measured_traffic():
    try:
        with open(TRAFFIC_PROFILE) as f:
            for line in f:
                if line.startswith("DRAM traffic per launch (read + write):"):
                    return float(line.split(":")[1].split()[0]) * 1e6
    except OSError:
        pass
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device=None):
    """Largest value of x over all ranks of the process group (the job's
    time is that of its slowest replica); x itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, n, ms_per_step):
    """Whole-job particle-updates/s: every rank advances its own replica of
    n particles by one iteration per step."""
    return ws * n / (ms_per_step * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"smc_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        try:
            for line in open(self.path):
                v = [x.strip() for x in line.split(",")]
                if len(v) >= 6 and v[0].isdigit():
                    rows.append(v)
        except Exception:
            return None
        if not rows:
            return None
        sm = sorted(int(r[0]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": int(rows[0][1]), "reasons": sorted(reasons),
                "samples": len(rows)}


def run_ours(args):
    import torch
    from paper_1306_5583_b300 import smc, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T_OBS, seed=0, **p)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n = args.n

    def make(scheme):
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme=scheme, threshold=0.5, seed=1 + rank,
                              max_data=T_OBS, max_records=T_OBS + 1, cv=p, keep_cdf=False)
        s = smc.Sampler(cfg, stream=stream, device=dev)
        s.set_data(y)
        return s

    def timed(scheme, K, W):
        """K timed SMC iterations (one captured-graph replay each) with the
        L2 flushed before each, then K event-timed launches of the fused
        move/weight kernel alone (the dominant kernel, for the roofline)."""
        s = make(scheme)
        with torch.cuda.stream(stream):
            s.initialize()
            s.iterate(W)
            stream.synchronize()
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
            if ws > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize(dev)
            t_wall = time.perf_counter()
            for h in range(HEAD_START):
                flush.fill_(float(-h))
            for k in range(K):
                if s.iteration() + 1 >= T_OBS:
                    s.initialize()
                flush.fill_(float(k))
                ev[k][0].record(stream)
                s.iterate(1)
                ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
            t_wall = time.perf_counter() - t_wall
            step_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
            hist = s.history(min(K + W + 1, T_OBS))
            frac_res = float(np.mean([r["resampled"] for r in hist[-K:]]))
            # the dominant kernel alone
            mv = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
            for h in range(HEAD_START):
                flush.fill_(float(-h))
            for k in range(K):
                if s.iteration() + 1 >= T_OBS:
                    s.initialize()
                flush.fill_(float(k))
                mv[k][0].record(stream)
                s.move()
                mv[k][1].record(stream)
                s.resample()
            torch.cuda.synchronize(dev)
            move_ms = [mv[k][0].elapsed_time(mv[k][1]) for k in range(K)]
            # the move kernel as it runs inside the replayed iteration graph:
            # two events captured immediately around it (read after each step)
            gb, ga = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.set_move_events(gb, ga)
            graph_move_ms = []
            for k in range(-W, K):
                if s.iteration() + 1 >= T_OBS:
                    s.initialize()
                flush.fill_(float(k))
                s.iterate(1)
                torch.cuda.synchronize(dev)
                if k >= 0:
                    graph_move_ms.append(gb.elapsed_time(ga))
            s.set_move_events(None, None)
        s.close()
        return dict(step_ms=step_ms, move_ms=move_ms, graph_move_ms=graph_move_ms, wall_s=t_wall,
                    resample_frac=frac_res)

    def full_run(scheme):
        """The whole filter of T = 1000 observations as one smc_iterate(999)
        on the replayed graph, CUDA events around it (no L2 flush between its
        iterations: the run as a user makes it)."""
        s = make(scheme)
        with torch.cuda.stream(stream):
            s.initialize()
            s.iterate(1)  # captures the graph
            s.initialize()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.iterate(T_OBS - 1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            lz = s.log_evidence()
        s.close()
        return {"iterations": T_OBS - 1, "ms": ms, "us_per_iteration": ms * 1e3 / (T_OBS - 1),
                "particle_updates_per_s": n * (T_OBS - 1) / (ms * 1e-3), "log_evidence": lz}

    headline = args.scheme
    with Clocks(local) as clk:
        main = timed(headline, args.steps, args.warmup)
    clocks = clk.summary()
    per_scheme = {}
    for sc in args.schemes.split(","):
        r = main if sc == headline else timed(sc, args.steps, args.warmup)
        per_scheme[sc] = dict(
            particle_updates_per_s=n / (np.mean(r["step_ms"]) * 1e-3),
            ms_per_step=float(np.mean(r["step_ms"])),
            move_us=float(np.mean(r["graph_move_ms"]) * 1e3),
            move_us_standalone=float(np.mean(r["move_ms"]) * 1e3),
            resample_fraction=r["resample_frac"])
        if sc == headline:
            per_scheme[sc]["full_run_T1000"] = full_run(sc)
    total_ms = max_over_ranks(float(np.sum(main["step_ms"])), dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(ws, n, ms_per_step)

    # dominant kernel: the fused move/weight kernel, timed by events captured
    # around it in the iteration graph (the standalone launch, bracketed by
    # events on the stream, adds the launch latency: reported beside it)
    move_us = float(np.mean(main["graph_move_ms"]) * 1e3)
    move_us_standalone = float(np.mean(main["move_ms"]) * 1e3)
    peak, peak_kind = measured_peaks()
    achieved = PF_BYTES_PER_PARTICLE * n / (move_us * 1e-6) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": measured_traffic(), "kernel": "pf_iterate_kernel<float, 0>",
                "kernel_us": round(move_us, 2),
                "kernel_timing": "mean over the timed steps of CUDA events captured immediately before and after the "
                                 "move kernel in the iteration graph (L2 flushed before each step); a standalone "
                                 f"launch bracketed by events on the stream: {move_us_standalone:.2f} us",
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                                  "profiles/pf_iterate_cv_gather_2e20.md (cold-cache capture; writes stay in L2)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.4 TB/s"}

    # the whole iteration (move kernel, resampler and launch gaps) against the
    # same peak: expected algorithmic bytes per particle-update over the
    # event-timed step
    f_res = main["resample_frac"]
    it_bytes = PF_BYTES_PER_PARTICLE + RESAMPLE_BYTES_PER_PARTICLE * f_res
    it_achieved = it_bytes * n / (ms_per_step * 1e-3) / 1e9
    roofline["iteration"] = {"achieved": round(it_achieved, 1), "frac": round(it_achieved / peak, 4),
                             "bytes_per_particle": round(it_bytes, 2),
                             "definition": "(40 B + 12 B x resample fraction) x N / ms_per_step: the whole "
                                           "iteration, kernels plus launch and completion gaps"}

    # end to end through the C ABI with host buffers (pinned): H2D of the
    # step's observation, D2H of the step's record
    e2e = run_e2e(make, headline, args.steps, max(3, args.warmup), y, dev, stream, flush) if rank == 0 else None
    launches = args.steps * (1 + RESAMPLE_KERNELS[headline])  # kernels of this library in the timed region
    out = {
        "metric": METRIC, "value": value, "unit": "particle-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_particles": n, "scheme": headline, "threshold": 0.5,
                   "l2": "1 GB buffer written between timed iterations (untimed)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "resample_fraction": main["resample_frac"]},
        "roofline": roofline,
        "per_scheme": per_scheme,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "device": device_summary(dev),
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(n, 8)
        if not args.no_extra:
            out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(n, 8)
            out["cpu_baseline"]["other_configs"] = oracle_baselines()
    if rank == 0 and not args.no_extra:
        extra = {}
        mufu = mufu_peak(dev)
        extra["mufu_peak_measured"] = mufu
        extra["pf_fp64_n1000_T100"] = bench_pf_fp64_small(dev, stream)
        extra["gmm_rw_n2^16"] = bench_gmm(dev, stream, mufu, move="rw")
        extra["gmm_mala_n2^18"] = bench_gmm(dev, stream, mufu, n=1 << 18, move="mala")
        extra["gmm_rw_vs_mala_n2^18"] = bench_gmm_accuracy(dev, stream, seeds=args.gmm_seeds)
        extra["pf_grad_n2^18_T500"] = bench_pf_grad(dev, stream)
        extra["batched_256"] = bench_batched(dev, stream)
        out["extra"] = extra
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def device_summary(dev):
    """The GPU the numbers come from, read at run time: name, SM count and
    L2 size (the flush writes FLUSH_BYTES between timed iterations)."""
    import torch
    pr = torch.cuda.get_device_properties(dev)
    l2 = int(getattr(pr, "L2_cache_size", 0))
    return {"name": pr.name, "sms": int(pr.multi_processor_count), "l2_bytes": l2,
            "flush_over_l2": round(FLUSH_BYTES / l2, 2) if l2 else None}


def run_e2e(make, scheme, K, W, y, dev, stream, flush):
    """K host-buffer iterations through smc_iterate_host, each timed on the
    host around the call (which synchronises), after W untimed ones (the
    first call of a context also captures its iteration graph)."""
    import torch
    from paper_1306_5583_b300 import smc
    s = make(scheme)
    obs = torch.empty(2, dtype=torch.float64, pin_memory=True)
    rec = torch.empty(ctypes.sizeof(smc.Record), dtype=torch.uint8, pin_memory=True)
    L = smc.lib()
    # the call's three arguments, marshalled once (the buffers stay the same)
    ctx = s.ctx
    obs_p = ctypes.c_void_p(obs.data_ptr())
    rec_p = ctypes.cast(ctypes.c_void_p(rec.data_ptr()), ctypes.POINTER(smc.Record))
    with torch.cuda.stream(stream):
        s.initialize()
        torch.cuda.synchronize(dev)
        total = 0.0
        steps = 0
        per_call = []
        for k in range(-W, K):
            t = s.iteration() + 1
            if t >= T_OBS:
                s.initialize()
                torch.cuda.synchronize(dev)
                t = 1
            obs.copy_(torch.from_numpy(y[t]))
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc = L.smc_iterate_host(ctx, obs_p, rec_p)
            dt = time.perf_counter() - t0
            smc.check(rc, "smc_iterate_host")
            if k >= 0:
                total += dt
                steps += 1
                per_call.append(dt)
    s.close()
    # host -> device per step: the observation (2 float64) and its flag word, read from the
    # context's mapped pinned staging by the first kernel of the call's graph; device -> host:
    # the step's record, written there by the move kernel (the error word only on an error),
    # and the call's sequence number, written by the graph's last kernel
    return {"value": s.n * steps / total, "unit": "particle-updates/s", "h2d_bytes_per_step": 16 + 4,
            "d2h_bytes_per_step": ctypes.sizeof(smc.Record) + 4,
            "timing": f"host wall clock per call, {W} untimed calls first; one graph launch per call, the "
                      "observation and the record through mapped pinned memory, the call returning when the "
                      "graph's last kernel has written its sequence number there; the call's ctypes arguments "
                      "built once before the loop",
            "per_call_us": {"p50": round(float(np.percentile(per_call, 50)) * 1e6, 1),
                            "p90": round(float(np.percentile(per_call, 90)) * 1e6, 1),
                            "max": round(float(np.max(per_call)) * 1e6, 1)}}


def mufu_peak(dev):
    """The special-function pipe's measured issue rate (smc_mufu_rate, a
    kernel of independent ex2 / lg2 chains), in MUFU operations per second,
    with the SM clock sampled while it ran."""
    from paper_1306_5583_b300 import smc
    import torch
    torch.cuda.synchronize(dev)
    with Clocks(dev.index if dev.index is not None else 0) as clk:
        rates = {kind: max(smc.mufu_rate(k, 8, 1 << 14)[0] for _ in range(5))
                 for k, kind in enumerate(("ex2_lg2", "ex2", "lg2"))}
    c = clk.summary() or {}
    mhz = c.get("sm_mhz") or 2032
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    per_clk = {k: v / (sms * mhz * 1e6) for k, v in rates.items()}
    # the GMM likelihood is almost all ex2 (n r per datum against n / 8 lg2):
    # its roofline is the ex2 rate
    return {"ops_per_s": rates["ex2"], "ops_per_s_by_kind": rates, "ops_per_clk_per_sm_by_kind": per_clk,
            "sm_mhz": mhz, "sms": sms,
            "how": "smc_mufu_rate: 8 blocks/SM x 256 threads x 8 independent chains of ex2.approx and/or "
                   "lg2.approx, 2^14 rounds, best of 5 event-timed launches per kind; the peak used is ex2's"}


def bench_gmm(dev, stream, mufu, n=1 << 16, T=500, move="rw", K=20):
    """GMM tempered sampler (Sec. 5.2): iterations per second and the MUFU
    roofline of the mcmc kernel, plus both evidence estimates of a full
    run.  The algorithmic count is the method's: per particle and iteration
    each Metropolis block evaluates n r exponentials and n logarithms
    (3 blocks: 15 000 for n = 1000, r = 4); a Langevin move evaluates the
    likelihood and its gradient once (n r + n).  The kernel itself folds
    eight logarithms into one (n / 8), which the implementation count
    reports beside it."""
    import torch
    from paper_1306_5583_b300 import smc, workloads
    y = workloads.gmm_data(1000, seed=0)
    mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA}[move]
    cfg = smc.make_config(model="gmm", n=n, precision=32, scheme="systematic", threshold=0.5, seed=1, max_data=1000,
                          max_records=T + 1, keep_cdf=False, gmm=dict(n_comp=4, n_iter=T, power=5.0, move=mv,
                                                                       mala_step=0.05))
    s = smc.Sampler(cfg, stream=stream, device=dev)
    s.set_data(y)
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(1)  # captures the iteration graph
        s.initialize()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.iterate(T)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        full_ms = e0.elapsed_time(e1)
        ds, ps = s.log_evidence(), s.path_sampling()
        # the mcmc kernel alone, late in the schedule (alpha near 1)
        s.initialize()
        s.iterate(T - K - 1)
        mk = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
        for k in range(K):
            s.move()
            s.resample()
            mk[k][0].record(stream)
            s.mcmc()
            mk[k][1].record(stream)
        torch.cuda.synchronize(dev)
        mcmc_ms = float(np.median([a.elapsed_time(b) for a, b in mk]))
    s.close()
    nd, r = 1000, 4
    algo = n * (3 * nd * (r + 1) if move == "rw" else nd * (r + 1))
    impl = n * (3 * nd * (r + 1.0 / 8) if move == "rw" else nd * (r + 1 + 1.0 / 8))
    rate = algo / (mcmc_ms * 1e-3)
    return {"n_particles": n, "iterations": T, "move": move, "ms_full_run": full_ms,
            "particle_updates_per_s": n * T / (full_ms * 1e-3), "log_evidence_standard": ds,
            "log_evidence_path_sampling": ps, "mcmc_kernel_us": mcmc_ms * 1e3,
            "mufu_ops_per_particle_iteration_algorithmic": algo / n,
            "mufu_ops_per_particle_iteration_kernel": impl / n,
            "mufu_ops_per_s_algorithmic": rate,
            "mufu_frac_of_measured_peak": rate / mufu["ops_per_s"],
            "mufu_frac_of_measured_peak_kernel_count": impl / (mcmc_ms * 1e-3) / mufu["ops_per_s"]}


def bench_gmm_accuracy(dev, stream, n=1 << 18, T=500, seeds=8):
    """The random-walk and Langevin samplers at the same N: mean and
    standard deviation of both evidence estimates over seeds, the
    event-timed run, and the time each needs to reach the smaller of the two
    standard deviations (replicates averaged: time x (sd / sd_common)^2)."""
    import torch
    from paper_1306_5583_b300 import smc, workloads
    y = workloads.gmm_data(1000, seed=0)
    out = {}
    for move in ("rw", "mala"):
        mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA}[move]
        ds, ps, ms = [], [], []
        for seed in range(seeds):
            cfg = smc.make_config(model="gmm", n=n, precision=32, scheme="systematic", threshold=0.5, seed=100 + seed,
                                  max_data=1000, max_records=T + 1, keep_cdf=False,
                                  gmm=dict(n_comp=4, n_iter=T, power=5.0, move=mv, mala_step=0.05))
            s = smc.Sampler(cfg, stream=stream, device=dev)
            s.set_data(y)
            with torch.cuda.stream(stream):
                s.initialize()
                s.iterate(1)
                s.initialize()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.iterate(T)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
                ds.append(s.log_evidence())
                ps.append(s.path_sampling())
            s.close()
        out[move] = {"log_evidence_standard_mean": float(np.mean(ds)), "log_evidence_standard_sd": float(np.std(ds, ddof=1)),
                     "log_evidence_path_mean": float(np.mean(ps)), "log_evidence_path_sd": float(np.std(ps, ddof=1)),
                     "ms_per_run": float(np.mean(ms))}
    sd_common = min(out["rw"]["log_evidence_standard_sd"], out["mala"]["log_evidence_standard_sd"])
    for move in ("rw", "mala"):
        o = out[move]
        o["ms_to_common_sd"] = o["ms_per_run"] * (o["log_evidence_standard_sd"] / sd_common) ** 2
    out["n_particles"] = n
    out["seeds"] = seeds
    out["common_sd"] = sd_common
    return out


def bench_batched(dev, stream, count=256):
    """256 filters of uneven N and T in one launch per kernel per
    iteration, against the same 256 filters run one by one through the plain
    API.  Both arms are timed by CUDA events on one stream around the
    iteration work only: every plain context is created, given its data and
    has its iteration graph captured before the timed region, which then
    holds each filter's initialize + iterate(T_b - 1); the batched arm holds
    the batch's initialize + run after the autotuner."""
    import torch
    from paper_1306_5583_b300 import smc, workloads
    ns, ts = workloads.batch_shapes(count, seed=0)
    p = dict(workloads.CV_DEFAULT)
    data = [workloads.cv_data(int(T), seed=1 + b, **p)[1] for b, T in enumerate(ts)]
    work = float(np.sum(ns.astype(np.float64) * ts))
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.5, seed=3,
                          max_data=int(ts.max()), keep_cdf=False, cv=p)
    bt = smc.Batch(cfg, ns, ts, stream=stream, device=dev)
    for b in range(count):
        bt.set_data(b, data[b])
    with torch.cuda.stream(stream):
        shape = bt.tune()
        bt.run()  # the iteration graph is captured here
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.initialize()
        bt.run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        batch_ms = e0.elapsed_time(e1)
        lz_batch = bt.log_evidence()
    bt.close()
    plain = []
    with torch.cuda.stream(stream):
        for b in range(count):
            pc = smc.make_config(model="cv", n=int(ns[b]), precision=32, scheme="systematic", threshold=0.5, seed=3,
                                 stream_id=b, max_data=int(ts[b]), keep_cdf=False, cv=p)
            s = smc.Sampler(pc, stream=stream, device=dev)
            s.set_data(data[b])
            s.initialize()
            if int(ts[b]) > 1:
                s.iterate(1)  # captures the context's iteration graph
            plain.append(s)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for b, s in enumerate(plain):
            s.initialize()
            s.iterate(int(ts[b]) - 1)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = e0.elapsed_time(e1)
        lz_plain = np.array([s.log_evidence() for s in plain])
    for s in plain:
        s.close()
    return {"filters": count, "particle_updates": work, "batched_ms": batch_ms,
            "batched_particle_updates_per_s": work / (batch_ms * 1e-3), "plain_one_by_one_ms": plain_ms,
            "plain_particle_updates_per_s": work / (plain_ms * 1e-3), "speedup": plain_ms / batch_ms,
            "autotuned": {"blocks_per_sm": shape[0], "tiles_per_item": shape[1]},
            "timing": "CUDA events around initialize + all iterations in both arms; contexts, data and graphs "
                      "prepared before the timed region",
            "log_evidence_identical": bool(np.array_equal(lz_batch, lz_plain))}


def bench_pf_grad(dev, stream, n=1 << 18, T=500):
    """Config 3b: the gradient of the log-likelihood estimate (the reverse
    sweep with recomputation over a recorded forward run) against the plain
    forward run, both CUDA-event timed after a warm-up (graph capture and
    first-launch costs outside the timed region)."""
    import torch
    from paper_1306_5583_b300 import smc, workloads
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T, seed=0, **p)
    out = {}

    def ev():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for rec in (False, True):
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme="systematic", threshold=0.5, seed=1, max_data=T,
                              cv=p, keep_cdf=False, record=rec, checkpoint_every=16)
        s = smc.Sampler(cfg, stream=stream, device=dev)
        s.set_data(y)
        with torch.cuda.stream(stream):
            s.initialize()
            s.iterate(T - 1)
            if rec:
                s.pf_grad()
            torch.cuda.synchronize(dev)
            e0, e1 = ev()
            e0.record(stream)
            s.initialize()
            s.iterate(T - 1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out["forward_recorded_ms" if rec else "forward_ms"] = e0.elapsed_time(e1)
            if rec:
                e0, e1 = ev()
                e0.record(stream)
                g = s.pf_grad()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                out["gradient_ms"] = e0.elapsed_time(e1)
                out["gradient"] = [float(v) for v in g]
        s.close()
    out["gradient_over_forward"] = out["gradient_ms"] / out["forward_ms"]
    out["gradient_plus_recorded_forward_over_forward"] = (out["gradient_ms"] + out["forward_recorded_ms"]) / out["forward_ms"]
    out["n_particles"] = n
    out["iterations"] = T
    return out


def bench_pf_fp64_small(dev, stream, T=100, n=1000, reps=5):
    """The FP64 particle filter at the paper's example size
    (N = 1000, T = 100): device time per iteration of the replayed graph."""
    import torch
    from paper_1306_5583_b300 import smc, workloads
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=n, precision=64, scheme="systematic", threshold=0.5, seed=0, max_data=T, cv=p,
                          keep_cdf=False)
    s = smc.Sampler(cfg, stream=stream, device=dev)
    s.set_data(y)
    ms = []
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(1)
        for _ in range(reps):
            s.initialize()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.iterate(T - 1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        lz = s.log_evidence()
    s.close()
    per_it = float(np.median(ms)) / (T - 1)
    return {"n_particles": n, "iterations": T, "precision": "f64", "us_per_iteration": per_it * 1e3,
            "particle_updates_per_s": n / (per_it * 1e-3), "log_evidence": lz,
            "bound": "launch latency (tiny N)"}


def cpu_baseline(n, iters):
    """The FP64 oracle on `iters` iterations at the full N (bounded sample),
    one process."""
    from oracle import cv as ocv
    from oracle import resample as ores
    from paper_1306_5583_b300 import workloads
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T_OBS, seed=0, **p)
    op = ocv.CVParams(**p)
    r = ocv.init_step(n, y[0], 1, op, 0.5)
    anc = ores.resample("systematic", r.lw, 1, 0) if r.resample else None
    t0 = time.perf_counter()
    for t in range(1, iters + 1):
        r = ocv.step(r.x, r.lw, r.L, anc, t, y[t], 1, op, 0.5)
        anc = ores.resample("systematic", r.lw, 1, t) if r.resample else None
    dt = time.perf_counter() - t0
    return {"value": n * iters / dt, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{iters} iterations of the same filter at N={n} (numpy float64 + exact integer "
                      f"resampling), single process"}


def _oracle_block_move(args):
    """One block of particles through the oracle's move and weight (a
    worker of the all-core baseline)."""
    from oracle import cv as ocv
    x_blk, base_blk, i0, t, y_t, seed, params = args
    op = ocv.CVParams(**params)
    idx = np.arange(i0, i0 + x_blk.shape[1])
    x = ocv.move(x_blk, t, seed, op, index=idx)
    return x, base_blk + ocv.loglik(x, y_t, op)


def cpu_baseline_all_cores(n, iters):
    """The same oracle, particle-parallel over every core the process may
    use (os.sched_getaffinity): the move and weight of each block of
    particles in a worker process (a spawn pool, started before any further
    GPU work), the normaliser, ESS test and exact integer resampling in the
    parent, as in the one-process run."""
    import multiprocessing as mp
    from oracle import cv as ocv
    from oracle import resample as ores
    from oracle import weights as ow
    from paper_1306_5583_b300 import workloads
    cores = len(os.sched_getaffinity(0))
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T_OBS, seed=0, **p)
    op = ocv.CVParams(**p)
    r = ocv.init_step(n, y[0], 1, op, 0.5)
    anc = ores.resample("systematic", r.lw, 1, 0) if r.resample else None
    x, lw, L = r.x, r.lw, r.L
    bounds = np.linspace(0, n, cores + 1).astype(np.int64)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_block_move, [(x[:, :8], np.zeros(8), 0, 1, y[1], 1, p)] * cores)  # workers warm
        t0 = time.perf_counter()
        for t in range(1, iters + 1):
            xs = x[:, anc] if anc is not None else x
            base = np.full(n, -math.log(n)) if anc is not None else lw - L
            parts = pool.map(_oracle_block_move, [(xs[:, a:b], base[a:b], int(a), t, y[t], 1, p)
                                                  for a, b in zip(bounds[:-1], bounds[1:])])
            x = np.concatenate([q[0] for q in parts], axis=1)
            lw = np.concatenate([q[1] for q in parts])
            _, L = ow.log_sum_exp(lw)
            W = np.exp(lw - L)
            res = ow.resample_decision(1.0 / float(np.sum(W * W)), n, 0.5)
            anc = ores.resample("systematic", lw, 1, t) if res else None
        dt = time.perf_counter() - t0
    return {"value": n * iters / dt, "unit": "particle-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{iters} iterations at N={n}: move and weight in {cores} spawned worker processes over "
                      f"particle blocks, normaliser and exact integer resampling in the parent"}


def oracle_baselines():
    """The FP64 oracle (numpy, one process) on bounded samples of the other
    workloads, in particle-updates per second: the FP64 filter at N = 1000,
    T = 100 in full; the GMM sampler (random-walk and Langevin moves) on one
    iteration at N = 2^12 late in the schedule (each particle-update costs
    the same at any N); the likelihood gradient on a recorded forward run
    plus its reverse sweep at N = 2^10, T = 50; the batched filters run the
    particle filter's arithmetic, whose rate the N = 2^20 filter's baseline
    gives."""
    from oracle import cv as ocv
    from oracle import gmm as ogmm
    from oracle import grad as ograd
    from oracle import resample as ores
    from paper_1306_5583_b300 import workloads
    p = dict(workloads.CV_DEFAULT)
    op = ocv.CVParams(**p)
    out = {}
    _, y = workloads.cv_data(100, seed=0, **p)
    t0 = time.perf_counter()
    ocv.run(y, 1000, 0, op, scheme="systematic", threshold=0.5)
    out["pf_fp64_n1000_T100"] = {"value": 1000 * 99 / (time.perf_counter() - t0), "sample": "the whole run"}
    yg = workloads.gmm_data(1000, seed=0)
    gp = ogmm.GMMParams(r=4, T=500, power=5.0)
    n = 1 << 12
    for move in ("rw", "mala"):
        st = ogmm.init_state(n, yg, 1, gp)
        t, a_t = 450, ogmm.alpha(450, gp)
        t0 = time.perf_counter()
        if move == "rw":
            ogmm.mcmc(st, a_t, t, yg, 1, gp)
        else:
            ogmm.mala_step(st, a_t, t, yg, 1, gp, eps=0.05)
        out[f"gmm_{move}"] = {"value": n / (time.perf_counter() - t0),
                              "sample": f"one {move} move of N = {n} at t = {t}, n = 1000, r = 4"}
    _, yc = workloads.cv_data(50, seed=0, **p)
    t0 = time.perf_counter()
    anc = ograd.base_run(yc, 1 << 10, 1, op)
    ograd.gradient(yc, 1 << 10, 1, op, anc)
    out["pf_grad"] = {"value": (1 << 10) * 50 / (time.perf_counter() - t0),
                      "sample": "recorded forward run and reverse sweep, N = 2^10, T = 50 (forward + gradient "
                                "per particle-update)"}
    return out


def run_reference(args):
    """The oracle as it stands on this host's cores: W untimed and K timed
    steps, each one oracle iteration of the same filter on a bounded sample
    of the workload (n_s particles, n_s chosen so that the K + W steps take
    about a minute; particle-updates/s is per particle, so the unit is the
    same as the full-size arm's)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import cv as ocv
    from oracle import resample as ores
    from paper_1306_5583_b300 import workloads
    K, W = args.steps, args.warmup
    n_s = 1 << 18
    while n_s > 4096 and n_s * (K + W) > 60e6:  # about 1e6 oracle particle-updates per second
        n_s >>= 1
    n_s = min(n_s, args.n)
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T_OBS, seed=0, **p)
    op = ocv.CVParams(**p)
    r = ocv.init_step(n_s, y[0], 1, op, 0.5)
    anc = ores.resample("systematic", r.lw, 1, 0) if r.resample else None
    t = 0
    total = 0.0
    for k in range(-W, K):
        t = t + 1 if t + 1 < T_OBS else 1
        t0 = time.perf_counter()
        r = ocv.step(r.x, r.lw, r.L, anc, t, y[t], 1, op, 0.5)
        anc = ores.resample("systematic", r.lw, 1, t) if r.resample else None
        if k >= 0:
            total += time.perf_counter() - t0
    value = n_s * K / total
    sample = (f"{K} timed iterations (after {W} untimed) of one filter at N={n_s} (numpy float64 + exact integer "
              f"resampling), single process")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-updates/s",
           "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": total * 1e3 / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_particles": args.n, "scheme": "systematic", "threshold": 0.5,
                      "oracle_sample_particles": n_s},
           "cpu_baseline": {"value": value, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", default="systematic")
    ap.add_argument("--n-particles", dest="n", type=int, default=N_FULL)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the GMM, batched and gradient sections")
    ap.add_argument("--schemes", default="systematic,stratified,multinomial,residual,residual_systematic,"
                                         "residual_stratified")
    ap.add_argument("--gmm-seeds", dest="gmm_seeds", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
