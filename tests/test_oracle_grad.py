"""Pins of the oracle's particle-filter gradient (stop-gradient resampling)."""
import numpy as np
import pytest

from oracle import cv, grad
from paper_1306_5583_b300 import workloads


@pytest.mark.parametrize("gaussian", [False, True])
def test_gradient_matches_central_differences(gaussian):
    p = cv.CVParams(gaussian_obs=gaussian)
    _, y = workloads.cv_data(12, seed=3, gaussian_obs=gaussian)
    n, seed = 512, 5
    anc = grad.base_run(y, n, seed, p, threshold=0.6)
    assert any(a is not None for a in anc) and any(a is None for a in anc)
    J, g = grad.gradient(y, n, seed, p, anc)
    fd = grad.finite_difference(y, n, seed, p, anc, h=1e-4)
    cmp = slice(0, 3) if gaussian else slice(0, 4)
    assert np.allclose(g[cmp], fd[cmp], rtol=2e-5, atol=1e-6), (g, fd)
    # the replayed estimate reproduces the base run
    recs, _ = cv.run(y, n, seed, p, threshold=0.6)
    assert abs(J - recs[-1]["logZ"]) < 1e-10


def test_gradient_detects_a_dropped_normaliser_term():
    """Power check: dropping the -W sum(gbar) term of the weight adjoint
    changes the gradient visibly (so the test above would catch it)."""
    p = cv.CVParams()
    _, y = workloads.cv_data(8, seed=4)
    n, seed = 256, 2
    anc = grad.base_run(y, n, seed, p, threshold=0.3)
    assert any(a is None for a in anc[:-1])
    _, g = grad.gradient(y, n, seed, p, anc)
    fd = grad.finite_difference(y, n, seed, p, anc, h=1e-4)
    import oracle.grad as m
    orig = m.gradient

    def broken(y, n, seed, p, ancestors):
        T = y.shape[0]
        J, xs, lws, Ls = m.replay(y, n, seed, p, ancestors)
        gg = np.zeros(4)
        gbar_next = None
        for t in range(T - 1, -1, -1):
            W = np.exp(lws[t] - Ls[t])
            gbar = W if (t == T - 1 or ancestors[t] is not None) else W + gbar_next
            _, _, ds, _ = m.dloglik(xs[t], y[t], p)
            gg[2] += np.sum(gbar * ds)
            gbar_next = gbar
        return J, gg
    _, gb = broken(y, n, seed, p, anc)
    assert abs(gb[2] - fd[2]) > 100 * abs(g[2] - fd[2]) + 1e-3
