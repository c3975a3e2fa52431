"""GPU gradient of the particle filter's log-likelihood estimate (stop-gradient
resampling, noise fixed by its Philox counters) against the oracle's float64
reverse-mode gradient on the same (GPU-recorded) resampling, and against
central finite differences of the GPU's own replayed estimate."""
import numpy as np
import pytest

from gpu_common import cv_params, need_gpu, oracle_params, torch
from oracle import grad as ograd
from paper_1306_5583_b300 import smc, workloads


def _run(n, T, precision, model="cv", seed=3, threshold=0.6, ck=4):
    p = cv_params()
    _, y = workloads.cv_data(T, seed=2, gaussian_obs=(model == "cv_gauss"), **p)
    cfg = smc.make_config(model=model, n=n, precision=precision, scheme="systematic", threshold=threshold, seed=seed,
                          max_data=T, cv=p, keep_cdf=False, record=True, checkpoint_every=ck)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(T - 1)
    flags = [r["resampled"] for r in s.history(T)]
    anc = [s.ancestor_history(t).astype(np.int64) if flags[t] else None for t in range(T)]
    return s, y, oracle_params(p, model), anc


pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model", ["cv", "cv_gauss"])
def test_fp64_gradient_matches_oracle(model):
    need_gpu()
    n, T, seed = 1000, 11, 3
    s, y, op, anc = _run(n, T, 64, model=model, seed=seed, ck=4)
    assert any(a is not None for a in anc[:-1]) and any(a is None for a in anc[:-1])
    g = s.pf_grad()
    J, gref = ograd.gradient(y, n, seed, op, anc)
    assert abs(s.log_evidence() - J) < 1e-9
    k = 4 if model == "cv" else 3
    assert np.allclose(g[:k], gref[:k], rtol=1e-8, atol=1e-9), (g, gref)


def test_fp32_gradient_matches_oracle():
    need_gpu()
    n, T, seed = 1 << 14, 20, 5
    s, y, op, anc = _run(n, T, 32, seed=seed, ck=6)
    g = s.pf_grad()
    _, gref = ograd.gradient(y, n, seed, op, anc)
    assert np.allclose(g, gref, rtol=1e-4, atol=1e-4 * np.abs(gref).max()), (g, gref)
    th = np.array([op.sd_pos, op.sd_vel, op.obs_scale, op.obs_df])
    assert abs(s.pf_replay(th) - s.log_evidence()) < 1e-6 * abs(s.log_evidence())


def test_fp32_gradient_at_the_benchmarked_size():
    """N = 2^18 with a checkpoint every 16 iterations, the benchmarked
    launch configuration (T = 40 instead of 500 keeps the oracle's reverse
    sweep to seconds; three checkpoint segments, the last one ragged): the
    FP32 gradient and estimate against the oracle's float64 ones on the
    GPU-recorded resampling."""
    need_gpu()
    n, T, seed = 1 << 18, 40, 1
    s, y, op, anc = _run(n, T, 32, seed=seed, threshold=0.5, ck=16)
    assert any(a is not None for a in anc[:-1]) and any(a is None for a in anc[:-1])
    g = s.pf_grad()
    J, gref = ograd.gradient(y, n, seed, op, anc)
    assert abs(s.log_evidence() - J) < 1e-4 + 1e-6 * abs(J), (s.log_evidence(), J)
    assert np.allclose(g, gref, rtol=1e-4, atol=1e-4 * np.abs(gref).max()), (g, gref)


def test_fp64_gradient_matches_finite_differences_of_the_gpu_replay():
    """Central differences (h = 1e-3 relative) of the GPU's own replayed
    estimate, in float64 where the difference quotient is not dominated by
    rounding (in float32 the estimate's rounding, ~1e-6 relative of |log Z|,
    swamps a difference over a step of 2e-5 in sd_pos)."""
    need_gpu()
    n, T, seed = 4096, 15, 8
    s, y, op, anc = _run(n, T, 64, seed=seed, ck=5)
    g = s.pf_grad()
    th = np.array([op.sd_pos, op.sd_vel, op.obs_scale, op.obs_df])
    assert abs(s.pf_replay(th) - s.log_evidence()) < 1e-10
    for j in range(4):
        h = 1e-3 * th[j]
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (s.pf_replay(tp) - s.pf_replay(tm)) / (2 * h)
        assert abs(fd - g[j]) < 1e-4 * max(abs(g[j]), 1.0), (j, fd, g[j])


def test_gradient_is_deterministic_and_checkpoint_independent():
    need_gpu()
    a = _run(5000, 13, 32, ck=3)[0].pf_grad()
    b = _run(5000, 13, 32, ck=3)[0].pf_grad()
    c = _run(5000, 13, 32, ck=13)[0].pf_grad()
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)
