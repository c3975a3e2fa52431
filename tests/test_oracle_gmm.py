"""Pins of the oracle's Gaussian-mixture sampler (Sec. 5.2)."""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import gmm
from paper_1306_5583_b300 import workloads


def _theta(n, r, seed):
    g = np.random.default_rng(seed)
    mu = g.normal(scale=3, size=(r, n))
    lam = g.gamma(2.0, 1.0, size=(r, n))
    om = g.dirichlet(np.ones(r), size=n).T
    return mu, lam, om


def test_log_lik_matches_enumeration_over_allocations():
    """exp l(theta) = sum over allocations z of prod_k omega_{z_k} N(y_k | mu_{z_k}, 1/lambda_{z_k})."""
    y = np.array([-1.3, 0.2, 2.7, 0.9, -0.4])
    for r in (1, 2, 3):
        mu, lam, om = _theta(4, r, r)
        ll = gmm.log_lik(mu, lam, om, y)
        for i in range(4):
            tot = 0.0
            for z in itertools.product(range(r), repeat=len(y)):
                term = 1.0
                for k, j in enumerate(z):
                    term *= om[j, i] * stats.norm.pdf(y[k], mu[j, i], 1 / math.sqrt(lam[j, i]))
                tot += term
            assert abs(ll[i] - math.log(tot)) < 1e-10


def test_log_lik_far_off_means_stay_finite():
    y = workloads.gmm_data(100, seed=1)
    mu = np.array([[500.0], [-700.0]])
    lam = np.array([[3.0], [0.5]])
    om = np.array([[0.5], [0.5]])
    ll = gmm.log_lik(mu, lam, om, y)
    assert np.isfinite(ll).all()


def test_log_prior_matches_scipy():
    p = gmm.GMMParams(r=3, mu0=0.5, sd0=10.0, shape0=2, rate0=1.5)
    mu, lam, om = _theta(6, 3, 7)
    lp = gmm.log_prior(mu, lam, om, p)
    for i in range(6):
        ref = (stats.norm.logpdf(mu[:, i], 0.5, 10.0).sum() + stats.gamma.logpdf(lam[:, i], 2, scale=1 / 1.5).sum()
               + stats.dirichlet.logpdf(om[:, i], np.ones(3)))
        assert abs(lp[i] - ref) < 1e-10


def test_prior_draws_have_the_prior_law():
    p = gmm.GMMParams(r=4, shape0=2, rate0=2.0)
    y = workloads.gmm_data(50, seed=0)
    s = gmm.init_state(20000, y, 3, p)
    assert stats.kstest(s.mu[1], stats.norm(p.mu0, p.sd0).cdf).pvalue > 1e-4
    assert stats.kstest(s.lam[2], stats.gamma(2, scale=0.5).cdf).pvalue > 1e-4
    assert stats.kstest(s.om[0], stats.beta(1, 3).cdf).pvalue > 1e-4
    assert np.allclose(s.om.sum(axis=0), 1)


def test_metropolis_blocks_leave_the_prior_invariant():
    """At alpha = 0 every block targets the prior: the law of the chain
    stays the prior (a dropped Jacobian in the lambda or omega block fails)."""
    p = gmm.GMMParams(r=3)
    y = workloads.gmm_data(30, seed=2)
    s = gmm.init_state(20000, y, 5, p)
    for rnd in range(6):
        s, _ = gmm.mcmc(s, 0.0, 100 + rnd, y, 5, p)
    assert stats.kstest(s.mu[0], stats.norm(0, 10).cdf).pvalue > 1e-4
    assert stats.kstest(s.lam[1], stats.expon().cdf).pvalue > 1e-4
    assert stats.kstest(s.om[2], stats.beta(1, 2).cdf).pvalue > 1e-4


def test_dropped_jacobian_would_be_detected():
    """The invariance test has power: the same chain without the lambda
    Jacobian drifts away from the prior."""
    p = gmm.GMMParams(r=2)
    y = workloads.gmm_data(10, seed=3)
    s = gmm.init_state(20000, y, 6, p)
    import oracle.gmm as mod
    for rnd in range(6):
        n = s.mu.shape[1]
        idx = np.arange(n)
        _, s_lam, _ = mod.proposal_scales(0.0)
        from oracle import philox
        z = s_lam * philox.normals(6, idx, 200 + rnd, philox.TAG_MH_LAMBDA, 2)
        lam = np.exp(np.log(s.lam) + z)
        lp = mod.log_prior(s.mu, lam, s.om, p)
        w = philox.draw_words(6, idx, 200 + rnd, philox.TAG_MH_LAMBDA, 0, philox.DRAW_MH_UNIFORM)
        acc = np.log(philox.uniform(w[:, 0])) <= lp - s.lprior      # no Jacobian
        s = mod.State(s.mu, np.where(acc, lam, s.lam), s.om, np.where(acc, lp, s.lprior), s.llik)
    assert stats.kstest(s.lam[0], stats.expon().cdf).pvalue < 1e-6


def _r1_log_evidence(y, p):
    """log p(y) for r = 1: mu integrated out (compound-symmetric normal),
    lambda by quadrature."""
    n = len(y)
    d = y - p.mu0
    S1, S2 = d.sum(), (d * d).sum()
    s2 = p.sd0 ** 2

    def logf(lam):
        logdet = -(n - 1) * math.log(lam) + math.log(1 / lam + n * s2)
        quad = lam * S2 - lam * lam * s2 * S1 * S1 / (1 + n * lam * s2)
        ll = -0.5 * n * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad
        lg = p.shape0 * math.log(p.rate0) - math.lgamma(p.shape0) + (p.shape0 - 1) * math.log(lam) - p.rate0 * lam
        return ll + lg

    grid = np.exp(np.linspace(-8, 4, 2001))
    m = max(logf(v) for v in grid)
    val, _ = integrate.quad(lambda u: math.exp(logf(math.exp(u)) - m + u), -12, 6, limit=500, epsabs=1e-13,
                            epsrel=1e-11)
    return m + math.log(val)


def test_r1_evidence_against_quadrature():
    p = gmm.GMMParams(r=1, T=60, power=4.0)
    g = np.random.default_rng(4)
    y = 1.0 + g.standard_normal(20)
    truth = _r1_log_evidence(y, p)
    ds, ps = [], []
    for seed in range(4):
        a, b, _ = gmm.run(y, 2000, seed, p)
        ds.append(a)
        ps.append(b)
    assert abs(np.mean(ds) - truth) < 0.05, (np.mean(ds), truth)
    assert abs(np.mean(ps) - truth) < 0.15, (np.mean(ps), truth)


def test_single_step_is_importance_sampling_from_the_prior():
    """T = 1: alpha goes 0 -> 1 at once and the standard estimate is
    log mean_i exp l(theta_i) over the prior draws."""
    p = gmm.GMMParams(r=2, T=1)
    y = workloads.gmm_data(40, seed=5)
    n, seed = 3000, 8
    ds, _, _ = gmm.run(y, n, seed, p)
    s0 = gmm.init_state(n, y, seed, p)
    m = s0.llik.max()
    assert abs(ds - (m + math.log(np.mean(np.exp(s0.llik - m))))) < 1e-10


def test_schedules():
    p = gmm.GMMParams(T=500, power=5.0)
    assert gmm.alpha(0, p) == 0.0 and gmm.alpha(500, p) == 1.0
    assert abs(gmm.alpha(250, p) - 0.5 ** 5) < 1e-15
    pl = gmm.GMMParams(T=10, schedule="linear")
    assert abs(gmm.alpha(3, pl) - 0.3) < 1e-15
    assert gmm.proposal_scales(1.0) == (0.15, 0.3, 0.4)
    assert gmm.proposal_scales(0.0) == gmm.proposal_scales(0.02)


def test_mala_gradient_matches_central_differences():
    p = gmm.GMMParams(r=3, shape0=2, rate0=1.5)
    y = workloads.gmm_data(60, seed=8)
    mu, lam, om = _theta(5, 3, 11)
    u = gmm.to_unconstrained(mu, lam, om)
    for a_t in (0.0, 0.3, 1.0):
        g, _ = gmm.grad_log_target_u(u, a_t, y, p)
        h = 1e-5
        for k in range(u.shape[0]):
            up, um = u.copy(), u.copy()
            up[k] += h
            um[k] -= h
            fd = (gmm.log_target_u(up, a_t, y, p) - gmm.log_target_u(um, a_t, y, p)) / (2 * h)
            assert np.allclose(g[k], fd, rtol=1e-6, atol=1e-5), (a_t, k, g[k], fd)


def test_mala_leaves_the_prior_invariant():
    p = gmm.GMMParams(r=3)
    y = workloads.gmm_data(30, seed=2)
    s = gmm.init_state(20000, y, 9, p)
    accs = []
    for rnd in range(8):
        s, acc = gmm.mala_step(s, 0.0, 300 + rnd, y, 9, p, eps=0.5)
        accs.append(acc.mean())
    assert 0.05 < np.mean(accs) < 0.99
    assert stats.kstest(s.mu[0], stats.norm(0, 10).cdf).pvalue > 1e-4
    assert stats.kstest(s.lam[1], stats.expon().cdf).pvalue > 1e-4
    assert stats.kstest(s.om[2], stats.beta(1, 2).cdf).pvalue > 1e-4


def test_moves_at_slots_equal_the_same_particles_of_the_whole_system():
    """mh_block and mala_step with explicit slots (the Philox counter index
    of each particle) give exactly the rows of the whole system's move at
    those slots: a particle's move depends on its own slot only."""
    p = gmm.GMMParams(r=3)
    y = workloads.gmm_data(40, seed=1)
    s = gmm.init_state(300, y, 4, p)
    sub = np.array([0, 7, 8, 150, 299])
    a_t = 0.3
    for block in ("mu", "lambda", "weight"):
        whole, acc_w, d_w, u_w = gmm.mh_block(s, block, a_t, 5, y, 4, p, return_delta=True)
        part, acc_p, d_p, u_p = gmm.mh_block(s.take(sub), block, a_t, 5, y, 4, p, return_delta=True, slots=sub)
        assert np.array_equal(part.mu, whole.mu[:, sub]) and np.array_equal(part.om, whole.om[:, sub])
        assert np.array_equal(d_p, d_w[sub]) and np.array_equal(u_p, u_w[sub]) and np.array_equal(acc_p, acc_w[sub])
    whole, acc_w, d_w, u_w = gmm.mala_step(s, a_t, 6, y, 4, p, eps=0.05, return_delta=True)
    part, acc_p, d_p, u_p = gmm.mala_step(s.take(sub), a_t, 6, y, 4, p, eps=0.05, return_delta=True, slots=sub)
    assert np.array_equal(part.lam, whole.lam[:, sub]) and np.array_equal(d_p, d_w[sub])
    assert np.array_equal(acc_p, acc_w[sub])
    # the default slots are 0 .. n - 1
    same, _ = gmm.mh_block(s, "mu", a_t, 5, y, 4, p, slots=np.arange(300))
    assert np.array_equal(same.mu, gmm.mh_block(s, "mu", a_t, 5, y, 4, p)[0].mu)


def test_adaptive_alpha_two_point_closed_form():
    """Uniform W and l_i in {0, -c} (half each): CESS(delta) =
    N (1 + u)^2 / (2 (1 + u^2)) with u = exp(-c delta), so CESS = rho N at
    u = ((1 - 2 rho) root of (1 - 2 rho) u^2 + 2 u + (1 - 2 rho) = 0); the
    bisection lands on that delta, CESS(0) = N, and a constant likelihood
    (CESS = N for every delta) jumps straight to alpha = 1."""
    n, c = 1000, 37.0
    logW = np.full(n, -math.log(n))
    ll = np.where(np.arange(n) % 2 == 0, 0.0, -c)
    assert abs(gmm.log_cess(logW, ll, 0.0) - math.log(n)) < 1e-12
    for rho in (0.75, 0.9, 0.6):
        A = 1 - 2 * rho
        u = (-2 + math.sqrt(4 - 4 * A * A)) / (2 * A)   # the root in (0, 1)
        delta = -math.log(u) / c
        a_prev = 0.125
        a = gmm.adaptive_alpha(logW, ll, a_prev, rho)
        assert abs((a - a_prev) - delta) < 1e-9, (rho, a - a_prev, delta)
        assert abs(gmm.log_cess(logW, ll, a - a_prev) - math.log(rho * n)) < 1e-8
    assert gmm.adaptive_alpha(logW, np.full(n, -3.0), 0.25, 0.5) == 1.0
    assert gmm.adaptive_alpha(logW, ll, 1.0, 0.5) == 1.0


def test_adaptive_schedule_r1_evidence_against_quadrature():
    """The CESS-targeted schedule as a whole: alpha increases to 1 within
    the iteration cap, the standard estimate matches the r = 1 quadrature
    value (the same bar as the fixed schedule), and the path-sampling
    estimate, whose trapezoid rule is biased on a coarse alpha grid,
    approaches it as the CESS target (and so the number of steps) grows."""
    g = np.random.default_rng(4)
    y = 1.0 + g.standard_normal(20)
    truth = _r1_log_evidence(y, gmm.GMMParams(r=1))
    ds, ps_err, steps = [], {}, {}
    for rho in (0.8, 0.99):
        p = gmm.GMMParams(r=1, T=400, schedule="adaptive", ess_target=rho)
        errs = []
        for seed in range(3 if rho == 0.8 else 1):
            a, b, recs = gmm.run(y, 2000, seed, p)
            al = [r.alpha for r in recs]
            assert all(x2 >= x1 for x1, x2 in zip(al, al[1:])) and al[-1] == 1.0
            steps[rho] = sum(1 for x in al if x < 1.0)
            if rho == 0.8:
                ds.append(a)
            errs.append(abs(b - truth))
        ps_err[rho] = float(np.mean(errs))
    assert abs(np.mean(ds) - truth) < 0.05, (np.mean(ds), truth)
    assert steps[0.8] < steps[0.99] < 400
    assert ps_err[0.99] < 0.15 and ps_err[0.99] < ps_err[0.8], ps_err
