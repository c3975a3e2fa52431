"""Pin of the fixed-point resamplers to the plain definition of Sec. 2.1.

The oracle's resamplers (and the CUDA path, bit for bit) select ancestors on
exact fixed-point weights q_i = floor(w_i 2^F), w_i = exp(lw_i - max lw).  The
plain definition selects on the float64 CDF of the real weights w_i
(``resample.plain_resample``).  Both must give the same ancestors except for
outputs whose target lies within the two representations' error of a CDF
boundary:

* fixed point: Q_i / Q_N differs from S_i / S_N (S the exact partial sums of
  the float64 w) by at most N / (2^F S_N - N), because each floor loses less
  than one unit and the weights are at most 1;
* float64: the cumulative sum and the scaled target carry at most
  (N + 4) 2^-52 relative to C_N.

Every mismatch is checked against that bound and the mismatches are counted.
A target falls within delta of one of the N boundaries with probability
about 2 delta N, so a vector of N outputs expects about 2 delta N^2
mismatches: below 0.2 at N = 2^16 with the worst-case float64 term, far
less with the typical one.  Over this test's 600 174 outputs per scheme the
count is 0 for all six schemes; the test allows 2.
"""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import resample as R

SCHEMES = ["systematic", "stratified", "multinomial", "residual", "residual_systematic", "residual_stratified"]


def _vectors():
    g = np.random.default_rng(20240611)
    out = []
    for n in (1, 2, 3, 7, 64, 1000, 4097, 1 << 14, 1 << 16):
        out.append(("normal0.5", g.normal(scale=0.5, size=n)))
        out.append(("normal3", g.normal(scale=3.0, size=n)))
        if n <= 4097:
            out.append(("normal12", g.normal(scale=12.0, size=n)))
            lw = g.normal(scale=1.0, size=n)
            lw[g.random(n) < 0.3] = -np.inf
            if not np.isfinite(lw).any():
                lw[0] = 0.0
            out.append(("zeros", lw))
            out.append(("heavy", -5.0 * g.exponential(size=n)))
            lw = np.full(n, -30.0)
            lw[n // 2] = 0.0
            out.append(("dominant", lw))
            out.append(("equal", np.zeros(n)))
    return out


VECTORS = _vectors()


def _delta(w):
    n = w.shape[0]
    F = R.frac_bits(n)
    S = math.fsum(w)
    return n / (2.0 ** F * S - n) + (n + 4) * 2.0 ** -52


def _targets(scheme, n, seed, t):
    k = np.arange(n, dtype=np.float64)
    if scheme == "systematic":
        return (k + (2 * philox.systematic_u24(seed, t) + 1) / 2.0 ** 25) / n
    js = np.asarray(philox.resample_u24(seed, t, n), dtype=np.float64)
    if scheme == "stratified":
        return (k + (2 * js + 1) / 2.0 ** 25) / n
    return np.sort((2 * js + 1) / 2.0 ** 25)


def _mismatches_within(a_fp, a_pl, C, p, delta):
    """Indices of differing outputs; each must have every CDF boundary between
    the two ancestors within delta of its target."""
    bad = np.flatnonzero(a_fp != a_pl)
    c = C / C[-1]
    for k in bad:
        lo, hi = sorted((int(a_fp[k]), int(a_pl[k])))
        gap = np.max(np.abs(c[lo:hi] - p[k]))
        assert gap <= delta, (k, lo, hi, gap, delta)
    return bad.size


def _check_plain(scheme, lw, seed, t):
    a_fp = R.resample(scheme, lw, seed, t)
    a_pl = R.plain_resample(scheme, lw, seed, t)
    w = R.plain_weights(lw)
    n = w.shape[0]
    assert a_pl.shape == (n,) and np.all(np.diff(a_pl) >= 0)
    assert not np.any(w[a_pl] == 0.0)
    if scheme not in R.RESIDUAL_STEPS:
        return _mismatches_within(a_fp, a_pl, np.cumsum(w), _targets(scheme, n, seed, t), _delta(w)), 0
    step = R.RESIDUAL_STEPS[scheme]
    # residual: the deterministic copies, then the multinomial residual draws
    q = R.quantise(lw)
    d_fp, R_fp, r_fp, s = R.residual_parts(q)
    d_pl, R_pl, r_pl = R.plain_residual_parts(w)
    S = math.fsum(w)
    F = R.frac_bits(n)
    QN = sum(int(v) for v in q)
    elem = n * n / (S * (2.0 ** F * S - n)) + n * 2.0 ** -51   # error of N W_i per particle
    if R_fp != R_pl or not np.array_equal(np.asarray(d_fp), d_pl):
        # a floor(N W_i) decision flipped: some N W_i lies within the error of an integer
        nw = n * w / S
        assert np.min(np.abs(nw - np.round(nw))[np.asarray(d_fp) != d_pl]) <= elem
        return 0, 1
    if R_fp == 0:
        assert np.array_equal(a_fp, a_pl)
        return 0, 0
    if step == "multinomial":
        P, D = R.multinomial_targets(R_fp, philox.resample_u24(seed, t, R_fp))
    elif step == "systematic":
        P, D = R.systematic_targets(R_fp, philox.systematic_u24(seed, t))
    else:
        P, D = R.stratified_targets(R_fp, philox.resample_u24(seed, t, R_fp))
    x_fp = R.select(R.cdf(r_fp), P, D)
    RC = np.cumsum(r_pl)
    p = R.plain_residual_targets(R_fp, seed, t, 0, step)
    x_pl = R.plain_select(RC, RC[-1] * p)
    eps = elem + 2.0 ** s / QN
    delta_res = 2 * n * eps / max(RC[-1] - n * eps, 1e-300) + (n + 4) * 2.0 ** -52
    m = _mismatches_within(x_fp, x_pl, RC, p, delta_res)
    if m == 0:
        assert np.array_equal(a_fp, a_pl)
    return m, 0


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fixed_point_ancestors_equal_the_plain_definition(scheme):
    """Over every weight vector (N = 1 ... 2^16, narrow, wide, heavy-tailed,
    with zero weights, one dominant particle, equal weights) and three
    iterations' uniforms: the fixed-point ancestors equal the plain real-weight
    ancestors except at outputs within the stated error of a boundary."""
    outputs = mism = flips = 0
    for v, (_, lw) in enumerate(VECTORS):
        for t in (0, 1, 2):
            m, f = _check_plain(scheme, lw, seed=17 + v, t=t)
            outputs += lw.shape[0]
            mism += m
            flips += f
    # bound on the counts: none expected at these sizes (see the module docstring)
    assert mism <= 2, mism
    assert flips == 0
    assert outputs > 100000


def test_plain_definition_catches_a_shifted_target():
    """The comparison has power: shifting the systematic targets by one
    output (a plausible off-by-one in k) breaks the equality, and the lower
    bound differs from the upper bound on ties."""
    g = np.random.default_rng(5)
    lw = g.normal(scale=1.0, size=512)
    C = np.cumsum(R.plain_weights(lw))
    a_fp = R.resample("systematic", lw, 3, 4)
    u = (2 * philox.systematic_u24(3, 4) + 1) / 2.0 ** 25
    k = np.arange(512)
    assert np.array_equal(R.plain_select(C, C[-1] * (k + u) / 512), a_fp)
    assert np.sum(R.plain_select(C, C[-1] * (k + 1 + u) / 512) != a_fp) > 100
    # ties (a target exactly on a boundary) go to the next particle
    C_eq = np.arange(1, 9, dtype=np.float64)
    assert np.array_equal(R.plain_select(C_eq, np.arange(8, dtype=np.float64)), np.arange(8))


@pytest.mark.parametrize("scheme", ["residual", "residual_systematic", "residual_stratified"])
def test_plain_residual_keeps_floor_copies_and_sums_to_n(scheme):
    g = np.random.default_rng(8)
    for n in (5, 97, 1000):
        lw = g.normal(scale=1.5, size=n)
        a = R.plain_resample(scheme, lw, 2, 7)
        w = R.plain_weights(lw)
        o = R.offspring(a, n)
        assert o.sum() == n
        assert np.all(o >= np.floor(n * w / w.sum()))
