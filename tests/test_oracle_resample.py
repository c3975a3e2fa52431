"""Pins of the oracle's resamplers: the replication counts R_i of Sec. 2.1
must sum to N and satisfy eq:resample (unbiasedness, E[R_i] = N W_i)."""
import math

import numpy as np
import pytest

from oracle import resample

LW6 = np.log(np.array([0.05, 0.3, 0.02, 0.33, 0.1, 0.2]))


def _W(lw):
    q = resample.quantise(lw)
    QN = sum(int(v) for v in q)
    return np.array([int(v) / QN for v in q])


def test_fixed_point_cdf_is_exact_and_bounded():
    g = np.random.default_rng(0)
    for n in (1, 2, 5, 1000, 1 << 12):
        lw = g.normal(scale=4, size=n)
        q = resample.quantise(lw)
        F = resample.frac_bits(n)
        assert max(int(v) for v in q) == 1 << F           # the max weight maps to 2^F
        Q = resample.cdf(q)
        assert int(Q[-1]) == sum(int(v) for v in q)
        assert int(Q[-1]) < 1 << 62
        W = np.exp(lw - lw.max())
        assert np.max(np.abs(np.array([int(v) for v in q], dtype=float) / 2.0 ** F - W)) <= 2.0 ** -F


@pytest.mark.parametrize("scheme", ["systematic", "stratified", "multinomial", "residual"])
def test_counts_sum_to_n_and_sorted(scheme):
    g = np.random.default_rng(1)
    for n in (1, 3, 17, 256):
        lw = g.normal(scale=2, size=n)
        a = resample.resample(scheme, lw, seed=5, t=3)
        assert a.shape == (n,)
        assert np.all(np.diff(a) >= 0)
        assert a.min() >= 0 and a.max() < n
        assert resample.offspring(a, n).sum() == n


@pytest.mark.parametrize("scheme", ["systematic", "stratified", "multinomial", "residual"])
def test_zero_weight_never_selected(scheme):
    lw = np.array([0.0, -np.inf, 1.0, -np.inf, -0.5, -np.inf, 2.0])
    for t in range(30):
        a = resample.resample(scheme, lw, seed=9, t=t)
        assert not np.isin(a, [1, 3, 5]).any()


def test_systematic_exact_unbiasedness_on_a_uniform_grid():
    """E over an evenly spaced grid of 4096 uniforms of the systematic
    counts equals N W_i up to the grid spacing (o_i is piecewise constant in
    u with at most one jump per stratum)."""
    n = 6
    q = resample.quantise(LW6)
    Q = resample.cdf(q)
    W = _W(LW6)
    G = 4096
    acc = np.zeros(n)
    for gidx in range(G):
        j = gidx * (1 << 24) // G + 977
        P, D = resample.systematic_targets(n, j)
        acc += resample.offspring(resample.select(Q, P, D), n)
    assert np.max(np.abs(acc / G - n * W)) <= 2 * n / G


def test_systematic_counts_are_floor_or_ceil():
    g = np.random.default_rng(2)
    for t in range(50):
        lw = g.normal(scale=1.5, size=40)
        W = _W(lw)
        o = resample.offspring(resample.resample("systematic", lw, 3, t), 40)
        assert np.all(o >= np.floor(40 * W) - 1e-9) and np.all(o <= np.ceil(40 * W) + 1e-9)


@pytest.mark.parametrize("scheme", ["stratified", "multinomial", "residual"])
def test_monte_carlo_unbiasedness(scheme):
    n = 6
    W = _W(LW6)
    M = 6000
    acc = np.zeros(n)
    acc2 = np.zeros(n)
    for t in range(M):
        o = resample.offspring(resample.resample(scheme, LW6, seed=11, t=t), n)
        acc += o
        acc2 += o * o
    mean = acc / M
    sd = np.sqrt(np.maximum(acc2 / M - mean ** 2, 1e-12) / M)
    assert np.all(np.abs(mean - n * W) <= 5 * sd + 1e-3), (mean, n * W, sd)


def test_multinomial_variance_is_binomial():
    """Multinomial counts have Var(R_i) = N W_i (1 - W_i); stratified ones
    are strictly less variable (a wrong scheme mix-up fails here)."""
    n = 6
    W = _W(LW6)
    M = 6000
    om = np.array([resample.offspring(resample.resample("multinomial", LW6, 4, t), n) for t in range(M)])
    os_ = np.array([resample.offspring(resample.resample("stratified", LW6, 4, t), n) for t in range(M)])
    vm = om.var(axis=0)
    target = n * W * (1 - W)
    assert np.all(np.abs(vm - target) < 0.12 * target + 0.02)
    assert os_.var(axis=0).sum() < 0.8 * vm.sum()


def test_residual_keeps_the_deterministic_part():
    g = np.random.default_rng(3)
    for t in range(30):
        lw = g.normal(scale=1.0, size=25)
        W = _W(lw)
        o = resample.offspring(resample.resample("residual", lw, 6, t), 25)
        assert np.all(o >= np.floor(25 * W + 1e-12))


def test_residual_parts_identity():
    g = np.random.default_rng(4)
    lw = g.normal(size=50)
    q = resample.quantise(lw)
    d, R, r, s = resample.residual_parts(q)
    QN = sum(int(v) for v in q)
    assert sum(d) + R == 50
    rem = [50 * int(v) - di * QN for v, di in zip(q, d)]
    assert sum(rem) == R * QN
    assert all(0 <= x < QN for x in rem)
    assert sum(r) < 1 << 62 and (R == 0 or sum(r) > 0)


def test_degenerate_single_particle_weight():
    lw = np.full(100, -np.inf)
    lw[42] = 0.0
    for scheme in ("systematic", "stratified", "multinomial", "residual"):
        a = resample.resample(scheme, lw, 1, 0)
        assert np.all(a == 42)


def test_equal_weights_systematic_is_identity():
    a = resample.resample("systematic", np.zeros(37), 8, 2)
    assert np.array_equal(a, np.arange(37))


RESIDUAL_VARIANTS = ["residual_systematic", "residual_stratified"]


@pytest.mark.parametrize("scheme", RESIDUAL_VARIANTS)
def test_residual_variants_keep_floor_copies_and_are_unbiased(scheme):
    """Douc et al.'s residual variants: floor(N W_i) copies always, counts
    sum to N, and E[R_i] = N W_i (Monte Carlo, 5 sigma)."""
    n = 6
    W = _W(LW6)
    M = 6000
    acc = np.zeros(n)
    acc2 = np.zeros(n)
    for t in range(M):
        o = resample.offspring(resample.resample(scheme, LW6, seed=12, t=t), n)
        assert o.sum() == n and np.all(o >= np.floor(n * W + 1e-12))
        acc += o
        acc2 += o * o
    mean = acc / M
    sd = np.sqrt(np.maximum(acc2 / M - mean ** 2, 1e-12) / M)
    assert np.all(np.abs(mean - n * W) <= 5 * sd + 1e-3), (mean, n * W, sd)


def test_residual_systematic_is_exactly_unbiased_on_a_uniform_grid():
    """With one uniform for all R residual outputs, the counts averaged over
    an evenly spaced grid of u equal N W_i up to the grid spacing, and each
    residual count is within one of R r_i / sum r (systematic property)."""
    n = 6
    q = resample.quantise(LW6)
    d, R, r, _ = resample.residual_parts(q)
    RQ = resample.cdf(r)
    W = _W(LW6)
    G = 4096
    acc = np.zeros(n)
    rs = sum(r)
    for gidx in range(G):
        j = gidx * (1 << 24) // G + 313
        P, D = resample.systematic_targets(R, j)
        extra = resample.offspring(resample.select(RQ, P, D), n)
        assert np.all(np.abs(extra - R * np.array(r, dtype=float) / rs) < 1.0 + 1e-9)
        acc += np.array(d) + extra
    assert np.max(np.abs(acc / G - n * W)) <= 2 * n / G


def test_stay_permutation_by_hand_and_invariants():
    """The in-place copy_from: a hand-worked case, then the invariants on
    random ancestor sets (same multiset, survivors in their own slot, the
    empty slots filled by the extra copies in increasing order)."""
    a = np.array([0, 0, 0, 2, 3, 3])
    # offspring 3, 0, 1, 2, 0, 0: slots 1, 4, 5 are empty; extras 0, 0, 3
    assert resample.stay_permutation(a).tolist() == [0, 0, 2, 3, 0, 3]
    g = np.random.default_rng(6)
    for n in (1, 2, 9, 500):
        for scheme in ("systematic", "multinomial", "residual"):
            anc = resample.resample(scheme, g.normal(scale=2.0, size=n), 1, int(g.integers(100)))
            p = resample.stay_permutation(anc)
            assert np.array_equal(np.sort(p), anc)
            o = resample.offspring(anc, n)
            assert np.all(p[o > 0] == np.flatnonzero(o > 0))
            assert np.all(np.diff(p[o == 0]) >= 0)
    assert resample.stay_permutation(np.arange(7)).tolist() == list(range(7))
