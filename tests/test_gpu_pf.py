"""GPU parity of the particle-filter hot path against the oracle, through
the C ABI (Algorithm 1 with every resampling scheme)."""
import math

import numpy as np
import pytest

from gpu_common import (SCHEMES, assert_close, check_resample, cv_params, make_pf, need_gpu, oracle_params,
                        step_and_check, torch)
from oracle import cv as ocv
from oracle import philox as ophilox
from oracle import resample as ores
from paper_1306_5583_b300 import smc, workloads

pytestmark = pytest.mark.gpu


def test_philox_matches_oracle_and_curand():
    need_gpu()
    import ctypes
    import os
    g = np.random.default_rng(0)
    ctr = g.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    key = [0xA4093822, 0x299F31D0]
    gpu = smc.philox4x32_10(ctr, key)
    ref = ophilox.philox4x32_10(ctr, key)
    assert np.array_equal(gpu, ref)
    # the CUDA toolkit's own Philox4x32-10 (curand device API) on the same input
    path = os.path.join(os.path.dirname(__file__), "gpu_support", "libcurand_philox.so")
    cl = ctypes.CDLL(path)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    do = torch.empty_like(dc)
    k = (ctypes.c_uint32 * 2)(*key)
    assert cl.curand_philox4x32_10(ctypes.c_void_p(dc.data_ptr()), k, ctypes.c_void_p(do.data_ptr()),
                                   ctypes.c_int64(ctr.shape[0])) == 0
    assert np.array_equal(do.cpu().numpy().view(np.uint32), ref)


@pytest.mark.parametrize("scheme,T,seed", [(sc, 40, 3) for sc in SCHEMES] + [("systematic", 100, 0)])
def test_fp64_filter_end_to_end(scheme, T, seed):
    """FP64, N = 1000 (the paper's example size): records, ancestors and the
    final particle system match the free-running oracle; the last case is
    the benchmarked run (T = 100, Philox key 0, data seed 0)."""
    need_gpu()
    n = 1000
    s, y, op = make_pf(n, T, 64, scheme=scheme, seed=seed)
    s.initialize()
    s.iterate(T - 1)
    recs = s.history(T)
    ref, last = ocv.run(y, n, seed, op, scheme=scheme, threshold=0.5)
    assert len(recs) == T
    for r, o in zip(recs, ref):
        assert r["t"] == o["t"]
        assert r["resampled"] == o["resampled"], r["t"]
        assert abs(r["L"] - o["L"]) < 1e-9
        assert abs(r["logZ"] - o["logZ"]) < 1e-9
        assert abs(r["ess"] - o["ess"]) < 1e-7 * n
        assert abs(r["mean_x"] - o["mean_x"]) < 1e-9 and abs(r["mean_y"] - o["mean_y"]) < 1e-9
    assert any(o["resampled"] for o in ref)
    assert_close(s.state(), last.x, 1e-10, "final state")
    assert_close(s.log_weight(), last.lw, 1e-10, "final log-weights")
    assert abs(s.log_evidence() - ref[-1]["logZ"]) < 1e-9


@pytest.mark.parametrize("n", [1, 63, 64, 65, 65536, 65537, 262144, 262145, (1 << 20) + 3])
def test_fp64_move_tiling_boundaries(n):
    """FP64 move tiles: one particle per thread, 64 threads per block up to
    N = 2^16 and 256 above; sizes on both sides of a tile and of the
    switch, ragged last tiles included, and on both sides of 1024 blocks,
    above which the last block combines the block partials in several
    passes; against the free-running oracle."""
    need_gpu()
    T, seed = 6, 7
    s, y, op = make_pf(n, T, 64, scheme="systematic", seed=seed, threshold=0.9)
    s.initialize()
    s.iterate(T - 1)
    recs = s.history(T)
    ref, last = ocv.run(y, n, seed, op, scheme="systematic", threshold=0.9)
    for r, o in zip(recs, ref):
        assert r["resampled"] == o["resampled"], r["t"]
        assert abs(r["logZ"] - o["logZ"]) < 1e-9
        assert abs(r["ess"] - o["ess"]) < 1e-9 * n
        assert abs(r["mean_x"] - o["mean_x"]) < 1e-9
    assert_close(s.state(), last.x, 1e-10, "final state")
    assert_close(s.log_weight(), last.lw, 1e-10, "final log-weights")


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n", [1, 3, 1000, 2049, 20000])
def test_fp32_teacher_forced_steps(scheme, n):
    """FP32 path: each iteration from the GPU's own previous particle system;
    states and log-weights within 1e-5, ancestors bit-exact."""
    need_gpu()
    T, seed = 8, 11
    s, y, op = make_pf(n, T, 32, scheme=scheme, seed=seed, threshold=0.9)
    s.initialize()
    r0 = s.history(1)[0]
    ref0 = ocv.init_step(n, y[0], seed, op, 0.9)
    assert_close(s.state(), ref0.x, 1e-5, "initial state")
    assert abs(r0["L"] - ref0.L) < 1e-4
    logz_gpu, logz_ref = r0["L"], ref0.L
    for t in range(1, T):
        rec, ref = step_and_check(s, y, op, t, seed, 32, 1e-5, scheme)
        logz_gpu += rec["L"]
        logz_ref += ref.L
    assert abs(logz_gpu - logz_ref) < 1e-4


@pytest.mark.parametrize("n", [1000, 4096])
def test_fp64_teacher_forced_steps(n):
    need_gpu()
    T, seed = 6, 5
    s, y, op = make_pf(n, T, 64, scheme="stratified", seed=seed, threshold=1.0)
    s.initialize()
    for t in range(1, T):
        step_and_check(s, y, op, t, seed, 64, 1e-11, "stratified")


def test_threshold_semantics():
    need_gpu()
    n, T = 2048, 6
    for thr, expect in ((1.0, True), (0.0, False), (-1.0, False), (2.0, True)):
        s, y, op = make_pf(n, T, 32, threshold=thr)
        s.initialize()
        s.iterate(T - 1)
        assert all(r["resampled"] == expect for r in s.history(T)), thr


def test_degenerate_weights_select_one_particle():
    """An observation far from every particle but one: all ancestors equal
    the argmax, for every scheme (q_i = 0 for the others)."""
    need_gpu()
    n = 4096
    for scheme in SCHEMES:
        s, y, op = make_pf(n, 3, 64, scheme=scheme, threshold=1.0, params=cv_params(obs_scale=1e-3, obs_df=1e6))
        s.initialize()
        lw = s.log_weight()
        anc = s.ancestors()
        assert np.all(anc == int(np.argmax(lw))), scheme


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_heavy_particles_in_some_tiles(scheme, precision):
    """Tiles where one particle owns hundreds of offspring beside tiles of
    ordinary weights, and a heavy particle in the ragged last tile: the
    ancestors are bit-exact against the oracle's selection rule on the
    GPU's CDF whichever way each tile is selected."""
    need_gpu()
    n, seed = 5 * 2048 + 777, 9
    s, y, op = make_pf(n, 2, precision, scheme=scheme, threshold=0.0, seed=seed)
    s.initialize()  # threshold 0: no resampling is pending
    g = np.random.default_rng(3)
    lw = g.normal(0.0, 0.5, n)
    for i, extra in ((2 * 2048 + 1001, 7.0), (3 * 2048 + 8, 5.5), (n - 3, 6.0)):
        lw[i] += extra  # N W_i of order 10^2 to 10^3
    s.write_log_weight(lw)
    lw_gpu = s.log_weight()
    s.resample(force=True)
    anc = check_resample(s, lw_gpu, 0, scheme, seed, precision)
    counts = np.bincount(anc, minlength=n)
    assert counts.max() > 64  # some tile spans several output windows


@pytest.mark.parametrize("scheme", SCHEMES)
def test_one_particle_owns_most_outputs(scheme):
    """One particle carries about 94 % of the weight: its tile owns some
    10^4 outputs, more than a block's shared-memory table of stratified
    draws (4096) and several selection windows; the ancestors are the
    oracle's on the GPU's CDF."""
    need_gpu()
    n, seed = 5 * 2048 + 777, 12
    s, y, op = make_pf(n, 2, 32, scheme=scheme, threshold=0.0, seed=seed)
    s.initialize()
    lw = np.random.default_rng(4).normal(0.0, 0.5, n)
    heavy = 3 * 2048 + 17
    lw[heavy] += 12.0
    s.write_log_weight(lw)
    lw_gpu = s.log_weight()
    s.resample(force=True)
    anc = check_resample(s, lw_gpu, 0, scheme, seed, 32)
    assert np.count_nonzero(anc == heavy) > 4096 + 2048


@pytest.mark.parametrize("scheme", ["systematic", "stratified"])
def test_boundaries_next_to_integers(scheme):
    """Equal weights give Q_i = (i + 1) 2^F, so every offspring boundary
    y_i = Q_i N / Q_N is an integer.  Systematic: z_i = y_i - c 2^-25 sits
    c 2^-25 below it, and a (seed, stream) whose draw makes c tiny puts
    every boundary inside the estimate's error margin.  Stratified: the
    fraction of y_i is 0, inside the margin.  Every decision then takes
    the exact branch; the selection rule gives the identity."""
    need_gpu()
    n = 1 << 22
    frac = 61 - 22
    found = None
    for seed in range(64):  # the oracle's Philox at t = 0 over all 16-bit stream ids
        ctr = np.zeros((65536, 4), dtype=np.uint64)
        ctr[:, 2] = ophilox.TAG_RESAMPLE | (np.arange(65536, dtype=np.uint64) << np.uint64(16))
        j = ophilox.u24(ophilox.philox4x32_10(ctr, ophilox.key_of(seed))[:, 0])
        hit = np.flatnonzero(j <= 63)
        if hit.size:
            found = (seed, int(hit[0]))
            break
    assert found is not None
    seed, stream = found
    assert ophilox.systematic_u24(seed, 0, stream) <= 63
    cfg = smc.make_config(model="cv", n=n, precision=32, scheme=scheme, threshold=0.0, seed=seed,
                          stream_id=stream, max_data=2, cv=cv_params())
    s = smc.Sampler(cfg)
    s.set_data(workloads.cv_data(2, seed=0, **cv_params())[1])
    s.initialize()
    s.write_log_weight(np.zeros(n))
    s.resample(force=True)
    Q = s.cdf()
    assert np.array_equal(Q, (np.arange(1, n + 1, dtype=np.uint64) << np.uint64(frac)))
    assert np.array_equal(s.ancestors(), np.arange(n, dtype=np.int32))
    s.close()


def test_nonfinite_weights_raise_and_leave_state():
    need_gpu()
    n, T = 1000, 5
    s, y, op = make_pf(n, T, 32)
    y = y.copy()
    y[2] = np.nan
    s.set_data(y)
    s.initialize()
    s.move()
    x1 = s.state()
    lw1 = s.log_weight()
    s.resample()
    s.move()  # NaN observation
    with pytest.raises(smc.SMCError) as e:
        s.sync()
    assert e.value.code == smc.E_NONFINITE
    # the previous particle system is still the current one
    with pytest.raises(smc.SMCError):
        s.state()
    s2_state = np.empty_like(x1)
    import ctypes
    rc = smc.lib().smc_read_state(s.ctx, s2_state.ctypes.data_as(ctypes.c_void_p), 0)
    assert rc == smc.E_NONFINITE
    assert np.array_equal(s2_state, x1)


def test_determinism_bit_identical():
    need_gpu()
    outs = []
    for _ in range(2):
        s, y, op = make_pf(30000, 12, 32, scheme="multinomial", seed=9)
        s.initialize()
        s.iterate(11)
        outs.append((s.state(), s.log_weight(), s.ancestors(), s.cdf(), s.log_evidence()))
    for a, b in zip(*outs):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_kalman_evidence_gaussian_variant():
    """FP32 GPU filter on the linear-Gaussian variant: the mean of Z-hat / Z
    over seeds is 1 within Monte Carlo error (unbiasedness, closed form)."""
    need_gpu()
    from oracle import kalman
    T, n, R = 25, 1 << 14, 24
    p = cv_params()
    _, y = workloads.cv_data(T, seed=2, gaussian_obs=True, **p)
    logz = kalman.kalman_loglik(y, oracle_params(p, "cv_gauss"))
    est = []
    for r in range(R):
        cfg = smc.make_config(model="cv_gauss", n=n, precision=32, seed=1000 + r, max_data=T, cv=p)
        s = smc.Sampler(cfg)
        s.set_data(y)
        s.initialize()
        s.iterate(T - 1)
        est.append(s.log_evidence())
    ratio = np.exp(np.array(est) - logz)
    assert abs(ratio.mean() - 1) < 5 * ratio.std(ddof=1) / math.sqrt(R) + 0.01


@pytest.mark.parametrize("scheme", SCHEMES)
def test_full_size_sampled(scheme):
    """N = 2^20 (the benchmarked size and launch configuration): sampled
    particles against the oracle's per-particle step, and ancestors of
    sampled slots by the exact selection rule on the GPU's CDF."""
    need_gpu()
    n, T, seed = 1 << 20, 6, 0
    s, y, op = make_pf(n, T, 32, scheme=scheme, seed=seed, threshold=1.0)
    s.initialize()
    g = np.random.default_rng(1)
    idx = np.sort(g.choice(n, size=2000, replace=False))
    for t in range(1, T):
        x_prev = s.state().astype(np.float64)
        lw_prev = s.log_weight().astype(np.float64)
        rec_prev = s.history(1)[0]
        anc = s.ancestors().astype(np.int64) if rec_prev["resampled"] else None
        s.move()
        x = s.state()
        lw = s.log_weight()
        # per-particle oracle on the sample: gather, move, weight
        src = anc[idx] if anc is not None else idx
        xp = x_prev[:, src]
        eps = ophilox.normals(seed, idx, t, ophilox.TAG_MOVE, 4)
        xm = np.stack([xp[0] + op.delta * xp[2] + op.sd_pos * eps[0], xp[1] + op.delta * xp[3] + op.sd_pos * eps[1],
                       xp[2] + op.sd_vel * eps[2], xp[3] + op.sd_vel * eps[3]])
        base = np.full(idx.size, -math.log(n)) if anc is not None else lw_prev[idx] - rec_prev["L"]
        assert_close(x[:, idx], xm, 1e-5, f"state t={t}")
        assert_close(lw[idx], base + ocv.loglik(xm, y[t], op), 1e-5, f"lw t={t}")
        s.resample()
        # CDF: exact prefix sums of non-negative integers
        Q = s.cdf()
        assert np.all(np.diff(Q.astype(np.float64)) >= 0)
        a = s.ancestors().astype(np.int64)
        assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < n
        if (scheme == "multinomial" or scheme.startswith("residual")) and t == 1:
            check_resample(s, lw, t, scheme, seed, 32)  # every output against the oracle
        if scheme == "multinomial":
            # output k: the first i with Q_i 2^25 > Q_N (2 j_(k) + 1), j_(k) the sorted draws
            import bisect
            QN = int(Q[-1])
            js = np.sort(ophilox.resample_u24(seed, t, n).astype(np.int64))
            Qlist = [int(v) for v in Q.astype(object)]
            for k in g.choice(n, size=300, replace=False):
                thr = (QN * (2 * int(js[k]) + 1)) >> 25
                assert a[k] == bisect.bisect_right(Qlist, thr)
        if scheme in ("systematic", "stratified"):
            QN = int(Q[-1])
            ks = g.choice(n, size=300, replace=False)
            js = ophilox.resample_u24(seed, t, n) if scheme == "stratified" else None
            jsys = ophilox.systematic_u24(seed, t)
            Ql = Q.astype(object)
            import bisect
            Qlist = [int(v) for v in Ql]
            for k in ks:
                j = jsys if scheme == "systematic" else int(js[k])
                thr = (QN * ((int(k) << 25) + 2 * j + 1)) // (n << 25)
                assert a[k] == bisect.bisect_right(Qlist, thr)
        else:
            # offspring counts sum to N and particles with zero weight have none
            q = np.diff(np.concatenate([[0], Q.astype(object)])).astype(object)
            zero = np.array([int(v) == 0 for v in q])
            assert not np.any(zero[a])


@pytest.mark.parametrize("scheme", ["multinomial", "residual", "residual_systematic", "residual_stratified"])
@pytest.mark.parametrize("n", [3 * (1 << 20) + 17, 5 * 2048 + 1])
def test_histogram_one_pass_sizes(scheme, n):
    """Multinomial and residual selection (by the draw histogram, or by the
    closed form over the residual outputs) where every block owns several
    weight tiles (N above one wave of tiles) and where most blocks own none:
    three forced resamplings in a row give the oracle's ancestors on the
    GPU's CDF, every output compared."""
    need_gpu()
    seed = 4
    s, y, op = make_pf(n, 4, 32, scheme=scheme, threshold=0.0, seed=seed)
    s.initialize()
    g = np.random.default_rng(5)
    for t in range(3):
        if t:
            s.move()  # the gather of the previous ancestors; iteration t
        s.write_log_weight(g.normal(0.0, 1.5, n))
        lw_gpu = s.log_weight()
        s.resample(force=True)
        check_resample(s, lw_gpu, t, scheme, seed, 32)
    s.close()


@pytest.mark.parametrize("scheme", ["residual", "residual_systematic", "residual_stratified"])
def test_residual_without_draws(scheme):
    """Equal weights at N = 2^k: every d_i = N q_i / Q_N = 1 exactly, so
    R = 0, no residual draws and the identity ancestors."""
    need_gpu()
    n = 1 << 16
    s, y, op = make_pf(n, 2, 32, scheme=scheme, threshold=0.0, seed=2)
    s.initialize()
    s.write_log_weight(np.zeros(n))
    s.resample(force=True)
    assert np.array_equal(s.ancestors(), np.arange(n, dtype=np.int32))
    s.close()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_bench_configuration_matches_cdf_path(scheme):
    """The benchmarked launch configuration (no stored CDF, whole iterations
    replayed from a CUDA graph, N = 2^20, ESS threshold 0.5) gives results
    bit-identical to the step-by-step path with the CDF stored, whose
    resampling the other tests check against the oracle."""
    need_gpu()
    n, T = 1 << 20, 12
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)
    outs = []
    for keep in (True, False):
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme=scheme, threshold=0.5, seed=3, max_data=T,
                              cv=p, keep_cdf=keep)
        stream = torch.cuda.Stream()
        s = smc.Sampler(cfg, stream=stream)
        s.set_data(y)
        with torch.cuda.stream(stream):
            s.initialize()
            if keep:
                for _ in range(T - 1):
                    s.move()
                    s.resample()
            else:
                s.iterate(T - 1)
        s.sync()
        outs.append((s.state(), s.log_weight(), s.ancestors(), s.log_evidence(),
                     [r["resampled"] for r in s.history(T)]))
        s.close()
    a, b = outs
    assert sum(a[4]) > 0
    for u, v in zip(a, b):
        assert np.array_equal(np.asarray(u), np.asarray(v))


def test_move_events_in_the_graph_change_nothing():
    """The profiling events recorded around the move kernel inside the
    iteration graph time a positive interval and leave every record and
    the particle system bit-identical."""
    need_gpu()
    n, T = 1 << 16, 8
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)
    outs = []
    for with_events in (False, True):
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme="systematic", threshold=0.7, seed=5,
                              max_data=T, cv=p, keep_cdf=False)
        stream = torch.cuda.Stream()
        s = smc.Sampler(cfg, stream=stream)
        s.set_data(y)
        with torch.cuda.stream(stream):
            s.initialize()
            if with_events:
                b, a = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.set_move_events(b, a)
            for _ in range(T - 1):
                s.iterate(1)
                if with_events:
                    stream.synchronize()
                    assert b.elapsed_time(a) > 0.0
        s.sync()
        outs.append((s.state(), s.log_weight(), [(r["L"], r["logZ"], r["resampled"]) for r in s.history(T)]))
        s.close()
    a0, a1 = outs
    assert np.array_equal(a0[0], a1[0]) and np.array_equal(a0[1], a1[1]) and a0[2] == a1[2]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_post_resampling_mean_fp64_matches_oracle(scheme):
    """SMC_FLAG_POST_MEAN: the record's post-resampling mean equals the
    oracle's (mean of the selected copies after a resampling step, the
    weighted mean otherwise), FP64, N = 1000, free-running."""
    need_gpu()
    n, T, seed = 1000, 30, 6
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=n, precision=64, scheme=scheme, threshold=0.5, seed=seed, max_data=T,
                          cv=p, post_mean=True)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(T - 1)
    recs = s.history(T)
    ref, _ = ocv.run(y, n, seed, oracle_params(p), scheme=scheme, threshold=0.5)
    assert any(o["resampled"] for o in ref) and not all(o["resampled"] for o in ref)
    for r, o in zip(recs, ref):
        assert r["resampled"] == o["resampled"]
        assert abs(r["post_mean_x"] - o["post_mean_x"]) < 1e-9, (r["t"], r["post_mean_x"], o["post_mean_x"])
        assert abs(r["post_mean_y"] - o["post_mean_y"]) < 1e-9
    s.close()


def test_post_resampling_mean_fp32_graph_and_host_call():
    """FP32 through the replayed graph and through smc_iterate_host: the
    post-resampling mean equals the mean of the GPU's own selected copies
    (1e-5), and without the flag the field is NaN."""
    need_gpu()
    n, T = 50000, 8
    p = cv_params()
    _, y = workloads.cv_data(T, seed=1, **p)
    stream = torch.cuda.Stream()
    for host in (False, True):
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme="systematic", threshold=1.0, seed=2,
                              max_data=T, cv=p, post_mean=True)
        s = smc.Sampler(cfg, stream=stream)
        s.set_data(y)
        with torch.cuda.stream(stream):
            s.initialize()
            for t in range(1, T):
                if host:
                    rec = s.iterate_host(y[t]).as_dict()
                else:
                    s.iterate(1)
                    rec = s.history(t + 1)[-1]
                stream.synchronize()
                x = s.state()
                a = s.ancestors().astype(np.int64)
                assert rec["resampled"]
                assert abs(rec["post_mean_x"] - float(np.mean(x[0][a].astype(np.float64)))) < 1e-5
                assert abs(rec["post_mean_y"] - float(np.mean(x[1][a].astype(np.float64)))) < 1e-5
        s.close()
    cfg = smc.make_config(model="cv", n=n, precision=32, scheme="systematic", threshold=1.0, seed=2, max_data=T,
                          cv=p)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(2)
    assert all(np.isnan(r["post_mean_x"]) for r in s.history(3))


@pytest.mark.parametrize("scheme", ["systematic", "multinomial", "residual_stratified"])
def test_inplace_ancestors_match_oracle(scheme):
    """SMC_FLAG_INPLACE: the step's ancestors in the in-place copy_from
    arrangement (survivors keep their slot) equal the oracle's arrangement of
    its own ancestors on the GPU's CDF, with heavy particles in several tiles
    and a ragged last tile; then an FP64 run with the arrangement matches
    the oracle filter run the same way."""
    need_gpu()
    n, seed = 5 * 2048 + 777, 9
    p = cv_params()
    _, y = workloads.cv_data(3, seed=0, **p)
    cfg = smc.make_config(model="cv", n=n, precision=32, scheme=scheme, threshold=0.0, seed=seed, max_data=3,
                          cv=p, inplace=True)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    g = np.random.default_rng(3)
    lw = g.normal(0.0, 0.7, n)
    for i, extra in ((2 * 2048 + 1001, 7.0), (3 * 2048 + 8, 5.5), (n - 3, 6.0)):
        lw[i] += extra
    s.write_log_weight(lw)
    lw_gpu = s.log_weight()
    s.resample(force=True)
    Qi = [int(v) for v in s.cdf().astype(object)]
    q_gpu = [Qi[0]] + [Qi[i] - Qi[i - 1] for i in range(1, n)]
    if scheme in ores.RESIDUAL_STEPS:
        ref = ores.residual(q_gpu, seed, 0, step=ores.RESIDUAL_STEPS[scheme])
    else:
        ref = {"systematic": ores.systematic, "multinomial": ores.multinomial}[scheme](Qi, seed, 0)
    anc = s.ancestors().astype(np.int64)
    assert np.array_equal(anc, ores.stay_permutation(ref))
    o = np.bincount(anc, minlength=n)
    assert np.count_nonzero(anc == np.arange(n)) == np.count_nonzero(o)
    s.close()
    # end to end in FP64
    T, n2 = 25, 1000
    _, y2 = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=n2, precision=64, scheme=scheme, threshold=0.5, seed=3, max_data=T, cv=p,
                          inplace=True)
    s = smc.Sampler(cfg)
    s.set_data(y2)
    s.initialize()
    s.iterate(T - 1)
    recs = s.history(T)
    ref_recs, last = ocv.run(y2, n2, 3, oracle_params(p), scheme=scheme, threshold=0.5, inplace=True)
    assert any(o["resampled"] for o in ref_recs)
    for r, o in zip(recs, ref_recs):
        assert r["resampled"] == o["resampled"]
        assert abs(r["logZ"] - o["logZ"]) < 1e-9
    assert_close(s.state(), last.x, 1e-10, "final state")
    s.close()
