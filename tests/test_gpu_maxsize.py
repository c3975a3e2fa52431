"""The largest particle filter a context takes: N = 2^30 particles, FP32.

At this size the whole arrays stay on the device (the readers' on-device
form, ``Sampler.read_device``); only sampled values come back to the host.
Checked, per iteration (Algorithm 1, every iteration resampling):
* sampled particles against the oracle's per-particle step (gather through
  the GPU's ancestors, the move with the oracle's Philox normals, the
  log-weight with the oracle's density), as in the N = 2^20 test;
* the record (log-normaliser, ESS, weighted means: Sec. 2.1's estimators)
  against float64 reductions of the GPU's own log-weights and states, so
  the move kernel's multi-pass combine of 2^20 block partials is checked
  at the largest grid;
* the fixed-point CDF non-decreasing and the ancestors sorted and in range,
  and sampled outputs k against the selection rule on the GPU's CDF:
  a_k is the first i with Q_i > the target of k, i.e.
  Q_{a_k - 1} <= target < Q_{a_k} (Q_{-1} = 0), which fixes a_k uniquely
  without the whole CDF on the host (systematic, stratified and, for the
  first step, multinomial).
"""
import math

import numpy as np
import pytest

from gpu_common import assert_close, make_pf, need_gpu, torch
from oracle import cv as ocv
from oracle import philox as ophilox

pytestmark = pytest.mark.gpu

N_MAX = 1 << 30


def _need_memory(nbytes):
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes:
        pytest.skip(f"needs {nbytes / 2**30:.0f} GiB of free device memory, {free / 2**30:.0f} GiB free")


def _host(t, idx):
    """t[..., idx] on the host (idx a numpy index array)."""
    return t[..., torch.as_tensor(idx, device=t.device)].cpu().numpy()


def _stratified_u24(seed, t, ks):
    """The 24-bit draws j_k of the sampled outputs ks only (word k % 4 of
    the oracle's call k // 4, as oracle.philox.resample_u24 takes them)."""
    ks = np.asarray(ks, dtype=np.int64)
    w = ophilox.draw_words(seed, ks // 4, t, ophilox.TAG_RESAMPLE, 0, 0)
    return ophilox.u24(w[np.arange(ks.size), ks % 4])


@pytest.mark.parametrize("scheme", ["systematic", "stratified"])
def test_maximum_size_sampled(scheme):
    need_gpu()
    n, T, seed = N_MAX, 3, 0
    _need_memory(120 << 30)  # the context (56 GiB), a state copy and float64 reductions
    s, y, op = make_pf(n, T, 32, scheme=scheme, seed=seed, threshold=1.0)
    try:
        s.initialize()
        g = np.random.default_rng(7)
        idx = np.sort(np.concatenate([g.choice(n, size=2000, replace=False), [0, n - 1]]))
        idx = np.unique(idx)
        for t in range(1, T):
            rec_prev = s.history(1)[0]
            assert rec_prev["resampled"]
            anc_d = s.read_device("ancestors")
            src = _host(anc_d, idx).astype(np.int64)
            del anc_d
            x_prev = s.read_device("state")
            xp = _host(x_prev, src).astype(np.float64)
            del x_prev
            s.move()
            # sampled particles: gather, move and weight of the oracle
            eps = ophilox.normals(seed, idx, t, ophilox.TAG_MOVE, 4)
            xm = np.stack([xp[0] + op.delta * xp[2] + op.sd_pos * eps[0],
                           xp[1] + op.delta * xp[3] + op.sd_pos * eps[1],
                           xp[2] + op.sd_vel * eps[2], xp[3] + op.sd_vel * eps[3]])
            x = s.read_device("state")
            lw = s.read_device("log_weight")
            assert_close(_host(x, idx), xm, 1e-5, f"state t={t}")
            assert_close(_host(lw, idx), -math.log(n) + ocv.loglik(xm, y[t], op), 1e-5, f"lw t={t}")
            # the record against float64 reductions of the same arrays
            rec = s.history(1)[0]
            assert rec["t"] == t
            lw64 = lw.double()
            L = float(torch.logsumexp(lw64, 0))
            W = torch.exp(lw64 - L)
            ess = 1.0 / float(torch.sum(W * W))
            mx = float(torch.sum(W * x[0].double()))
            my = float(torch.sum(W * x[1].double()))
            del lw64, W, x, lw
            assert abs(rec["L"] - L) <= 1e-6, (rec["L"], L)
            assert abs(rec["ess"] - ess) <= 1e-6 * ess, (rec["ess"], ess)
            assert abs(rec["mean_x"] - mx) <= 1e-6 * max(1.0, abs(mx)), (rec["mean_x"], mx)
            assert abs(rec["mean_y"] - my) <= 1e-6 * max(1.0, abs(my)), (rec["mean_y"], my)
            s.resample()
            Q = s.read_device("cdf")
            assert bool(torch.all(Q[1:] >= Q[:-1]))
            QN = int(Q[-1])
            a = s.read_device("ancestors")
            assert bool(torch.all(a[1:] >= a[:-1])) and int(a[0]) >= 0 and int(a[-1]) < n
            ks = np.unique(np.concatenate([g.choice(n, size=2000, replace=False), [0, n - 1]]))
            ak = _host(a, ks).astype(np.int64)
            hi = _host(Q, ak).astype(object)
            lo = np.where(ak > 0, _host(Q, np.maximum(ak - 1, 0)), 0).astype(object)
            del Q, a
            # the target of output k: Q_N (k + u_k) / N with u_k = (2 j + 1) 2^-25
            # (systematic: one j for every k; stratified: j_k per output)
            js = ([ophilox.systematic_u24(seed, t)] * ks.size if scheme == "systematic"
                  else [int(v) for v in _stratified_u24(seed, t, ks)])
            for k, j, a_k, q_lo, q_hi in zip(ks, js, ak, lo, hi):
                target = (QN * ((int(k) << 25) + 2 * j + 1)) // (n << 25)
                assert int(q_lo) <= target < int(q_hi), (scheme, t, int(k), int(a_k))
    finally:
        s.close()
        torch.cuda.empty_cache()


def test_maximum_size_multinomial():
    """Multinomial resampling of the first step at N = 2^30: about 64 draws
    per 24-bit value, so every bucket of the kernel's draw histogram takes
    its byte-count path.  Sampled outputs k against the rule
    a_k = the first i with Q_i > Q_N (2 j_(k) + 1) / 2^25 on the GPU's CDF,
    j_(k) the k-th smallest of the oracle's 2^30 draws (their histogram,
    from a spawned process pool started before the GPU work)."""
    import multiprocessing as mp
    import os

    import draw_hist

    need_gpu()
    n, seed = N_MAX, 0
    _need_memory(100 << 30)
    cores = max(1, min(16, len(os.sched_getaffinity(0))))
    with mp.get_context("spawn").Pool(cores) as pool:
        counts = draw_hist.draw_counts(seed, 0, n, pool, 4 * cores)
    assert counts.max() < 256  # no byte of the kernel's histogram wraps
    H = np.concatenate([[0], np.cumsum(counts)])  # H[v] = #{k : j_k < v}
    assert H[-1] == n
    s, y, op = make_pf(n, 2, 32, scheme="multinomial", seed=seed, threshold=1.0)
    try:
        s.initialize()  # the first move, then (always) resampling at t = 0
        assert s.history(1)[0]["resampled"]
        Q = s.read_device("cdf")
        assert bool(torch.all(Q[1:] >= Q[:-1]))
        QN = int(Q[-1])
        a = s.read_device("ancestors")
        assert bool(torch.all(a[1:] >= a[:-1])) and int(a[0]) >= 0 and int(a[-1]) < n
        g = np.random.default_rng(11)
        ks = np.unique(np.concatenate([g.choice(n, size=3000, replace=False), [0, n - 1]]))
        js = np.searchsorted(H, ks, side="right") - 1  # H[j] <= k < H[j + 1]: the k-th smallest draw
        ak = _host(a, ks).astype(np.int64)
        hi = _host(Q, ak).astype(object)
        lo = np.where(ak > 0, _host(Q, np.maximum(ak - 1, 0)), 0).astype(object)
        del Q, a
        for k, j, a_k, q_lo, q_hi in zip(ks, js, ak, lo, hi):
            target = (QN * (2 * int(j) + 1)) >> 25
            assert int(q_lo) <= target < int(q_hi), (int(k), int(j), int(a_k))
    finally:
        s.close()
        torch.cuda.empty_cache()
