"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI step by step and check each step against the oracle from the GPU's own
inputs (teacher forcing)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cv as ocv
from oracle import resample as ores
from paper_1306_5583_b300 import smc, workloads

SCHEMES = ["systematic", "stratified", "multinomial", "residual", "residual_systematic", "residual_stratified"]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def close(a, b, rel):
    """|a - b| <= rel * max(|b|, 1), elementwise."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) <= rel * np.maximum(np.abs(b), 1.0)


def assert_close(a, b, rel, what):
    ok = close(a, b, rel)
    if not np.all(ok):
        bad = np.flatnonzero(~np.asarray(ok).reshape(-1))
        a_ = np.asarray(a, dtype=np.float64).reshape(-1)
        b_ = np.asarray(b, dtype=np.float64).reshape(-1)
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {i}: gpu {a_[i]!r} oracle {b_[i]!r}")


def cv_params(model="cv", **kw):
    p = dict(workloads.CV_DEFAULT)
    p.update(kw)
    return p


def oracle_params(p, model="cv"):
    return ocv.CVParams(gaussian_obs=(model == "cv_gauss"), **p)


def make_pf(n, T, precision, scheme="systematic", threshold=0.5, seed=0, data_seed=0, model="cv", params=None):
    p = params or cv_params()
    _, y = workloads.cv_data(T, seed=data_seed, gaussian_obs=(model == "cv_gauss"), **p)
    cfg = smc.make_config(model=model, n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=T, cv=p)
    s = smc.Sampler(cfg)
    s.set_data(y)
    return s, y, oracle_params(p, model)


def check_resample(s, lw_gpu, t, scheme, seed, precision):
    """Ancestors bit-exact given the GPU's fixed-point CDF and the Philox
    uniforms; the GPU's fixed-point weights within rounding of the oracle's
    quantisation of the GPU's log-weights."""
    n = lw_gpu.shape[0]
    Q = s.cdf().astype(object)
    anc = s.ancestors().astype(np.int64)
    Qi = [int(v) for v in Q]
    q_gpu = [Qi[0]] + [Qi[i] - Qi[i - 1] for i in range(1, n)]
    q_ref = ores.quantise(lw_gpu.astype(np.float64))
    qg = np.array(q_gpu, dtype=np.float64)
    qr = np.array([float(v) for v in q_ref])
    tol = (4e-6 if precision == 32 else 1e-13) * qr + 2.0
    assert np.all(np.abs(qg - qr) <= tol), "fixed-point weights"
    if scheme in ores.RESIDUAL_STEPS:
        ref = ores.residual(q_gpu, seed, t, step=ores.RESIDUAL_STEPS[scheme])
    else:
        ref = {"systematic": ores.systematic, "stratified": ores.stratified,
               "multinomial": ores.multinomial}[scheme](Qi, seed, t)
    assert np.array_equal(anc, ref), f"ancestors at t={t} ({scheme}): {np.flatnonzero(anc != ref)[:5]}"
    return anc


def step_and_check(s, y, op, t, seed, precision, rel, scheme):
    """Teacher-forced check of iteration t >= 1 (move, weight, normalise)
    and of its resampling step."""
    x_prev = s.state().astype(np.float64)
    lw_prev = s.log_weight().astype(np.float64)
    rec_prev = s.history(1)[0]
    anc = s.ancestors().astype(np.int64) if rec_prev["resampled"] else None
    s.move()
    x = s.state().astype(np.float64)
    lw = s.log_weight()
    rec = s.history(1)[0]
    assert rec["t"] == t and rec["status"] == 0
    ref = ocv.step(x_prev, lw_prev, rec_prev["L"], anc, t, y[t], seed, op, 0.5)
    assert_close(x, ref.x, rel, f"state t={t}")
    assert_close(lw, ref.lw, rel, f"log-weights t={t}")
    assert_close(rec["L"], ref.L, 10 * rel, f"log-normaliser t={t}")
    assert_close(rec["ess"], ref.ess, 10 * rel, f"ESS t={t}")
    assert_close([rec["mean_x"], rec["mean_y"]], [ref.mean_x, ref.mean_y], 10 * rel, f"means t={t}")
    s.resample()
    if rec["resampled"]:
        check_resample(s, lw, t, scheme, seed, precision)
    return rec, ref
