"""Small, bounded workloads for kernel profiling (ncu captures of one kernel).

    python -m paper_1306_5583_b300.profile_case pf   --n 1048576 --iters 4 --threshold 1.0
    python -m paper_1306_5583_b300.profile_case step --n 1048576 --iters 4 --threshold 1.0
    python -m paper_1306_5583_b300.profile_case gmm  --n 65536 --iters 3 --move rw
    python -m paper_1306_5583_b300.profile_case gmm  --n 65536 --iters 3 --schedule adaptive
    python -m paper_1306_5583_b300.profile_case pf   --n 1048576 --iters 4 --scheme residual_systematic
    python -m paper_1306_5583_b300.profile_case pf   --n 1048576 --iters 4 --inplace
    python -m paper_1306_5583_b300.profile_case grad --n 262144 --iters 40
    python -m paper_1306_5583_b300.profile_case batch --count 64 --iters 20

Each case builds its inputs from the synthetic generators (workloads.py),
runs a few iterations through the C ABI and synchronises; it prints one
line.  The device footprint stays below a few GB.
"""
import argparse

import torch

from . import smc, workloads


def pf(a):
    p = dict(workloads.CV_DEFAULT)
    T = a.iters + 2
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=a.n, precision=32, scheme=a.scheme, threshold=a.threshold, seed=1,
                          max_data=T, cv=p, keep_cdf=False, inplace=a.inplace)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    for _ in range(a.iters):
        s.move()
        s.resample()
    return s.log_evidence()


def step(a):
    """Replayed iterations (smc_iterate on a non-default stream): the
    captured iteration graph the benchmark times."""
    p = dict(workloads.CV_DEFAULT)
    T = a.iters + 2
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=a.n, precision=32, scheme=a.scheme, threshold=a.threshold, seed=1,
                          max_data=T, cv=p, keep_cdf=False)
    stream = torch.cuda.Stream()
    s = smc.Sampler(cfg, stream=stream)
    s.set_data(y)
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(a.iters)
        stream.synchronize()
    return s.log_evidence()


def gmm(a):
    y = workloads.gmm_data(1000, seed=0)
    mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA, "rw_mala": smc.GMM_RW_MALA}[a.move]
    sched = {"prior": smc.ALPHA_PRIOR, "adaptive": smc.ALPHA_ADAPTIVE}[a.schedule]
    cfg = smc.make_config(model="gmm", n=a.n, precision=32, scheme="systematic", threshold=0.5, seed=1,
                          max_data=1000, max_records=a.iters + 2,
                          gmm=dict(n_comp=4, n_iter=500, move=mv, mala_step=0.05, schedule=sched))
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(a.iters)
    return s.log_evidence()


def grad(a):
    p = dict(workloads.CV_DEFAULT)
    T = a.iters
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=a.n, precision=32, seed=1, max_data=T, max_records=T, cv=p,
                          keep_cdf=False, record=True)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(T - 1)
    return float(s.pf_grad()[0])


def batch(a):
    ns, Ts = workloads.batch_shapes(count=a.count, seed=0)
    Ts = [min(int(t), a.iters) for t in Ts]
    p = dict(workloads.CV_DEFAULT)
    ys = [workloads.cv_data(t, seed=1 + b, **p)[1] for b, t in enumerate(Ts)]
    cfg = smc.make_config(model="cv", n=1024, precision=32, scheme="systematic", threshold=0.5, seed=1,
                          max_data=max(Ts), cv=p, keep_cdf=False)
    bt = smc.Batch(cfg, [int(v) for v in ns], Ts)
    for b, yb in enumerate(ys):
        bt.set_data(b, yb)
    bt.initialize()
    bt.run()
    return float(bt.log_evidence()[0])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["pf", "step", "gmm", "grad", "batch"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--threshold", type=float, default=1.0)
    ap.add_argument("--scheme", default="systematic")
    ap.add_argument("--move", default="rw")
    ap.add_argument("--schedule", default="prior", choices=["prior", "adaptive"])
    ap.add_argument("--inplace", action="store_true")
    ap.add_argument("--count", type=int, default=64)
    a = ap.parse_args()
    v = {"pf": pf, "step": step, "gmm": gmm, "grad": grad, "batch": batch}[a.case](a)
    torch.cuda.synchronize()
    print(f"{a.case} ok {v:.6f}")


if __name__ == "__main__":
    main()
