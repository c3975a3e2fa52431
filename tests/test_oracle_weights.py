"""Pins of the oracle's normaliser, ESS and resample test (Sec. 2.1)."""
import math

import numpy as np
import pytest

from oracle import weights


def test_normalised_sums_to_one_and_matches_naive():
    g = np.random.default_rng(0)
    lw = g.normal(size=1000)
    W = weights.normalised(lw)
    assert abs(W.sum() - 1) < 1e-14
    naive = np.exp(lw) / np.exp(lw).sum()
    assert np.max(np.abs(W - naive)) < 1e-15
    _, L = weights.log_sum_exp(lw)
    assert abs(L - math.log(np.exp(lw).sum())) < 1e-12


def test_shift_invariance_and_large_offsets():
    g = np.random.default_rng(1)
    lw = g.normal(size=100)
    W0 = weights.normalised(lw)
    W1 = weights.normalised(lw - 5000.0)       # would underflow without the shift
    assert np.max(np.abs(W0 - W1)) < 1e-12
    _, L0 = weights.log_sum_exp(lw)
    _, L1 = weights.log_sum_exp(lw - 5000.0)
    assert abs((L0 - 5000.0) - L1) < 1e-9


def test_ess_bounds_and_special_cases():
    n = 64
    assert abs(weights.ess(np.zeros(n)) - n) < 1e-9
    one = np.full(n, -np.inf)
    one[3] = 0.0
    assert abs(weights.ess(one) - 1) < 1e-12
    # k equal weights and the rest zero: ESS = k
    k = np.full(n, -np.inf)
    k[:10] = 2.5
    assert abs(weights.ess(k) - 10) < 1e-9
    g = np.random.default_rng(2)
    for _ in range(20):
        e = weights.ess(g.normal(scale=3, size=n))
        assert 1 - 1e-12 <= e <= n + 1e-9


def test_all_minus_inf_raises():
    with pytest.raises(FloatingPointError):
        weights.log_sum_exp(np.full(4, -np.inf))


def test_resample_decision():
    n = 100
    assert weights.resample_decision(100.0, n, 1.0)          # threshold >= 1: always
    assert not weights.resample_decision(1.0, n, 0.0)        # threshold <= 0: never
    assert weights.resample_decision(49.9, n, 0.5)
    assert not weights.resample_decision(50.0, n, 0.5)       # strict "<"


def test_previous_log_weight():
    lw = np.array([0.0, math.log(3.0)])
    _, L = weights.log_sum_exp(lw)
    b = weights.previous_log_weight(lw, L, False, 2)
    assert np.allclose(np.exp(b), [0.25, 0.75])
    assert np.allclose(weights.previous_log_weight(lw, L, True, 2), math.log(0.5))
