"""GPU parity of the Gaussian-mixture SMC sampler (Sec. 5.2, Algorithm 2)
against the oracle, through the C ABI."""
import math

import numpy as np
import pytest

from gpu_common import assert_close, check_resample, need_gpu, torch
from oracle import gmm as ogmm
from oracle import philox as ophilox
from oracle import resample as ores
from paper_1306_5583_b300 import smc, workloads

pytestmark = pytest.mark.gpu


def make_gmm(n, nd=1000, r=4, T=500, precision=32, scheme="systematic", threshold=0.5, seed=0, data_seed=0,
             schedule="prior", power=5.0, shape0=1, rate0=1.0, move="rw", eps=0.05, ess_target=0.5):
    y = workloads.gmm_data(nd, seed=data_seed)
    mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA, "rw_mala": smc.GMM_RW_MALA}[move]
    cfg = smc.make_config(model="gmm", n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=nd, max_records=T + 1,
                          gmm=dict(n_comp=r, n_iter=T, power=power, shape0=shape0, rate0=rate0, move=mv,
                                   mala_step=eps, ess_target=ess_target,
                                   schedule={"linear": smc.ALPHA_LINEAR, "prior": smc.ALPHA_PRIOR,
                                             "adaptive": smc.ALPHA_ADAPTIVE}[schedule]))
    s = smc.Sampler(cfg)
    s.set_data(y)
    op = ogmm.GMMParams(r=r, T=T, power=power, schedule=schedule, shape0=shape0, rate0=rate0, ess_target=ess_target)
    return s, y, op


def _tie_window(precision, a_t, ll_before, delta):
    """Near-tie window of a Metropolis decision log u <= delta: the FP32
    error of delta follows the magnitude of the tempered log-likelihoods it
    differences (a few float ulps of a_t |l| with |l| in the thousands, plus
    the rounding of the proposal itself), not |delta|; FP64 keeps a relative
    1e-9."""
    if precision == 64:
        return 1e-9 * np.maximum(1.0, np.abs(delta))
    return 2e-3 + 2e-6 * a_t * np.abs(ll_before)


def split_state(x, r):
    return x[:r], x[r:2 * r], x[2 * r:3 * r], x[3 * r], x[3 * r + 1]


def test_init_matches_oracle_fp64():
    need_gpu()
    n, r = 3000, 4
    s, y, op = make_gmm(n, nd=200, r=r, precision=64, seed=2)
    s.initialize()
    x = s.state()
    mu, lam, om, lp, ll = split_state(x, r)
    ref = ogmm.init_state(n, y, 2, op)
    assert_close(mu, ref.mu, 1e-12, "mu")
    assert_close(lam, ref.lam, 1e-12, "lambda")
    assert_close(om, ref.om, 1e-12, "omega")
    assert_close(lp, ref.lprior, 1e-12, "log-prior")
    assert_close(ll, ref.llik, 1e-11, "log-likelihood")
    rec = s.history(1)[0]
    assert abs(rec["path_u"] - ref.llik.mean()) < 1e-9 * abs(ref.llik.mean())
    assert abs(rec["ess"] - n) < 1e-6


@pytest.mark.parametrize("precision,r", [(64, 4), (32, 4), (32, 1), (32, 3), (32, 6)])
def test_teacher_forced_iterations(precision, r):
    """Each iteration from the GPU's own particle system: reweight,
    resampling (ancestors bit-exact on the GPU's CDF), the three Metropolis
    blocks (states within tolerance wherever no acceptance decision is a
    near tie) and the path-sampling integrand."""
    need_gpu()
    n, nd, T, seed = 4096 + 37, 300, 40, 5
    s, y, op = make_gmm(n, nd=nd, r=r, T=T, precision=precision, seed=seed, threshold=0.8)
    rel = 1e-11 if precision == 64 else 1e-5
    s.initialize()
    ties_total = 0
    for t in range(1, 7):
        x_prev = s.state().astype(np.float64)
        lw_prev = s.log_weight().astype(np.float64)
        rec_prev = s.history(1)[0]
        s.move()
        lw = s.log_weight()
        rec = s.history(1)[0]
        a_t, a_p = ogmm.alpha(t, op), ogmm.alpha(t - 1, op)
        ll_prev = x_prev[3 * r + 1]
        # lw_prev is normalised by its own log-sum-exp (or equal after a gather)
        base = lw_prev - ogmm.weights.log_sum_exp(lw_prev)[1]
        ref_lw = base + (a_t - a_p) * ll_prev
        assert_close(lw, ref_lw, rel, f"reweight t={t}")
        L_ref = ogmm.weights.log_sum_exp(ref_lw)[1]
        assert abs(rec["L"] - L_ref) < 10 * rel * max(1, abs(L_ref))
        assert abs(rec["alpha"] - a_t) < 1e-15
        s.resample()
        anc = None
        if rec["resampled"]:
            anc = check_resample(s, lw, t, "systematic", seed, precision)
        s.mcmc()
        x = s.state().astype(np.float64)
        src = anc if anc is not None else np.arange(n)
        xin = x_prev[:, src]
        mu, lam, om, lp, ll = split_state(xin, r)
        st = ogmm.State(mu.copy(), lam.copy(), om.copy(), lp.copy(), ll.copy())
        # recompute the cached values in float64 from the GPU's parameters
        st.lprior = ogmm.log_prior(st.mu, st.lam, st.om, op)
        st.llik = ogmm.log_lik(st.mu, st.lam, st.om, y)
        near = np.zeros(n, dtype=bool)
        for block in ("mu", "lambda", "weight") if r > 1 else ("mu", "lambda"):
            ll_before = st.llik.copy()
            st, acc, delta, logu = ogmm.mh_block(st, block, a_t, t, y, seed, op, return_delta=True)
            near |= np.abs(delta - logu) < _tie_window(precision, a_t, ll_before, delta)
        ok = ~near
        ties_total += int(near.sum())
        gm, gl, go, glp, gll = split_state(x, r)
        assert_close(gm[:, ok], st.mu[:, ok], rel, f"mu t={t}")
        assert_close(gl[:, ok], st.lam[:, ok], rel, f"lambda t={t}")
        assert_close(go[:, ok], st.om[:, ok], rel, f"omega t={t}")
        assert_close(glp[ok], st.lprior[ok], rel, f"log-prior t={t}")
        assert_close(gll[ok], st.llik[ok], rel, f"log-likelihood t={t}")
        rec = s.history(1)[0]
        # U_t from the GPU's own particles (weights after resampling are equal)
        lw_now = s.log_weight().astype(np.float64)
        W = np.exp(lw_now - ogmm.weights.log_sum_exp(lw_now)[1])
        assert abs(rec["path_u"] - np.sum(W * gll)) < 10 * rel * abs(rec["path_u"])
    assert ties_total < 0.01 * n * 6


def test_full_run_fp64_matches_oracle():
    """FP64, every iteration free-running on both sides: identical
    resampling decisions, standard and path-sampling estimates within 1e-8."""
    need_gpu()
    n, nd, r, T, seed = 2048, 100, 2, 30, 3
    s, y, op = make_gmm(n, nd=nd, r=r, T=T, precision=64, seed=seed)
    s.initialize()
    s.iterate(T)
    ds_ref, ps_ref, recs = ogmm.run(y, n, seed, op)
    gpu = s.history(T + 1)[1:]
    assert [g["resampled"] for g in gpu] == [o.resampled for o in recs]
    assert abs(s.log_evidence() - ds_ref) < 1e-8
    assert abs(s.path_sampling() - ps_ref) < 1e-8
    for g, o in zip(gpu, recs):
        assert abs(g["path_u"] - o.U) < 1e-8 * abs(o.U)
        assert np.allclose(g["accept"], o.accept, atol=2.0 / n)


def test_r1_evidence_against_quadrature_fp32():
    """FP32 GPU sampler on the r = 1 model: both estimators agree with the
    quadrature value of log p(y) within Monte Carlo error."""
    need_gpu()
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from test_oracle_gmm import _r1_log_evidence
    g = np.random.default_rng(4)
    y = 1.0 + g.standard_normal(20)
    op = ogmm.GMMParams(r=1, T=60, power=4.0)
    truth = _r1_log_evidence(y, op)
    ds, ps = [], []
    for seed in range(4):
        cfg = smc.make_config(model="gmm", n=1 << 14, precision=32, scheme="systematic", threshold=0.5, seed=seed,
                              max_data=20, max_records=61, gmm=dict(n_comp=1, n_iter=60, power=4.0))
        s = smc.Sampler(cfg)
        s.set_data(y)
        s.initialize()
        s.iterate(60)
        ds.append(s.log_evidence())
        ps.append(s.path_sampling())
    assert abs(np.mean(ds) - truth) < 0.03, (ds, truth)
    assert abs(np.mean(ps) - truth) < 0.1, (ps, truth)


def test_r1_ais_linear_schedule_against_quadrature_fp32():
    """Annealed importance sampling (threshold 0: the sampler never
    resamples) on the linear schedule alpha_t = t / T, r = 1: the standard
    estimate of log p(y) agrees with quadrature within Monte Carlo error.
    (The trapezoidal path-sampling estimate is biased on this schedule,
    which spends few steps where U(alpha) changes fastest; it is not
    checked here.)"""
    need_gpu()
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from test_oracle_gmm import _r1_log_evidence
    g = np.random.default_rng(4)
    y = 1.0 + g.standard_normal(20)
    op = ogmm.GMMParams(r=1, T=60, schedule="linear")
    truth = _r1_log_evidence(y, op)
    ds = []
    for seed in range(4):
        cfg = smc.make_config(model="gmm", n=1 << 14, precision=32, scheme="systematic", threshold=0.0, seed=seed,
                              max_data=20, max_records=61,
                              gmm=dict(n_comp=1, n_iter=60, schedule=smc.ALPHA_LINEAR))
        s = smc.Sampler(cfg)
        s.set_data(y)
        s.initialize()
        s.iterate(60)
        assert not any(r["resampled"] for r in s.history(61))
        ds.append(s.log_evidence())
    assert abs(np.mean(ds) - truth) < 0.05, (ds, truth)


def test_model_selection_over_component_counts():
    """The paper's use of the sampler: Bayesian comparison of mixture
    models by their evidence.  On data from four unit-variance components
    three standard deviations apart the log-evidence rises from r = 2 to
    3 to 4 (by about 29 and 9 nats at this size) and gains nothing beyond
    the true r; the margins leave room for the estimates' Monte Carlo
    error."""
    need_gpu()
    lz = {}
    for r in (2, 3, 4, 5):
        s, y, op = make_gmm(1 << 14, nd=1000, r=r, T=100, seed=7)
        s.initialize()
        s.iterate(100)
        lz[r] = s.log_evidence()
        s.close()
    assert lz[2] < lz[3] - 10 and lz[3] < lz[4] - 3, lz
    assert lz[5] < lz[4] + 3, lz


def test_benchmark_size_sampled():
    """N = 2^16, n = 1000, r = 4 (the benchmarked GMM workload, same launch
    configuration): a few iterations, sampled particles against the oracle."""
    need_gpu()
    n, r, seed = 1 << 16, 4, 0
    s, y, op = make_gmm(n, nd=1000, r=r, T=500, precision=32, seed=seed)
    s.initialize()
    g = np.random.default_rng(7)
    idx = np.sort(g.choice(n, size=512, replace=False))
    for t in range(1, 4):
        x_prev = s.state().astype(np.float64)
        s.move()
        rec = s.history(1)[0]
        s.resample()
        anc = s.ancestors().astype(np.int64) if rec["resampled"] else None
        s.mcmc()
        x = s.state().astype(np.float64)
        src = anc[idx] if anc is not None else idx
        mu, lam, om, lp, ll = split_state(x_prev[:, src], r)
        st = ogmm.State(mu.copy(), lam.copy(), om.copy(), ogmm.log_prior(mu, lam, om, op),
                        ogmm.log_lik(mu, lam, om, y))
        # per-particle oracle moves use the particle's own counter (its slot)
        near = np.zeros(idx.size, dtype=bool)
        a_t = ogmm.alpha(t, op)
        for block in ("mu", "lambda", "weight"):
            ll_before = st.llik.copy()
            st, acc, delta, logu = ogmm.mh_block(st, block, a_t, t, y, seed, op, return_delta=True, slots=idx)
            near |= np.abs(delta - logu) < _tie_window(32, a_t, ll_before, delta)
        ok = ~near
        gm, gl, go, glp, gll = split_state(x[:, idx], r)
        assert_close(gm[:, ok], st.mu[:, ok], 1e-5, f"mu t={t}")
        assert_close(gll[ok], st.llik[ok], 1e-5, f"l t={t}")
        assert near.sum() <= 10


@pytest.mark.parametrize("precision,move,r", [(64, "mala", 4), (32, "mala", 4), (32, "rw_mala", 3), (32, "mala", 1)])
def test_langevin_moves_teacher_forced(precision, move, r):
    """MALA (and random walk followed by MALA): the cached likelihood
    gradient equals the oracle's, and each move matches the oracle from the
    GPU's own particles wherever no decision is a near tie."""
    need_gpu()
    n, nd, T, seed, eps = 2048 + 19, 200, 30, 6, 0.05
    s, y, op = make_gmm(n, nd=nd, r=r, T=T, precision=precision, seed=seed, threshold=0.8, move=move, eps=eps)
    rel = 1e-10 if precision == 64 else 1e-5
    grel = 1e-9 if precision == 64 else 2e-4
    s.initialize()
    near_total = 0
    for t in range(1, 6):
        s.move()
        rec = s.history(1)[0]
        s.resample()
        anc = s.ancestors().astype(np.int64) if rec["resampled"] else None
        x_prev = s.state().astype(np.float64)
        src = anc if anc is not None else np.arange(n)
        xin = x_prev[:, src]
        mu, lam, om = xin[:r], xin[r:2 * r], xin[2 * r:3 * r]
        st = ogmm.State(mu.copy(), lam.copy(), om.copy(), ogmm.log_prior(mu, lam, om, op), ogmm.log_lik(mu, lam, om, y))
        if move == "mala":
            # cached gradient rows of the GPU against the oracle at the GPU's parameters
            _, gm, gl, gz = ogmm.loglik_grad(st.mu, st.lam, st.om, y)
            g_gpu = xin[3 * r + 2:]
            ref = np.concatenate([gm, gl, gz])
            assert_close(g_gpu, ref, grel * np.max(np.abs(ref)), f"cached gradient t={t}")
        a_t = ogmm.alpha(t, op)
        near = np.zeros(n, dtype=bool)
        if move == "rw_mala":
            for block in ("mu", "lambda", "weight") if r > 1 else ("mu", "lambda"):
                ll_before = st.llik.copy()
                st, acc, delta, logu = ogmm.mh_block(st, block, a_t, t, y, seed, op, return_delta=True)
                near |= np.abs(delta - logu) < _tie_window(precision, a_t, ll_before, delta)
        ll_before = st.llik.copy()
        st, acc, delta, logu = ogmm.mala_step(st, a_t, t, y, seed, op, eps=eps, return_delta=True)
        near |= np.abs(delta - logu) < _tie_window(precision, a_t, ll_before, delta)
        s.mcmc()
        x = s.state().astype(np.float64)
        ok = ~near
        near_total += int(near.sum())
        assert_close(x[:r][:, ok], st.mu[:, ok], rel, f"mu t={t}")
        assert_close(x[r:2 * r][:, ok], st.lam[:, ok], rel, f"lambda t={t}")
        assert_close(x[2 * r:3 * r][:, ok], st.om[:, ok], rel, f"omega t={t}")
        assert_close(x[3 * r + 1][ok], st.llik[ok], rel, f"log-likelihood t={t}")
        rec = s.history(1)[0]
        assert abs(rec["accept_mala"] - acc.mean()) <= (near.sum() + 1) / n
    assert near_total < 0.01 * n * 5


def test_mala_full_run_fp64_matches_oracle():
    need_gpu()
    n, nd, r, T, seed = 1024, 80, 2, 20, 4
    s, y, op = make_gmm(n, nd=nd, r=r, T=T, precision=64, seed=seed, move="mala", eps=0.1)
    s.initialize()
    s.iterate(T)
    ds_ref, ps_ref, recs = ogmm.run(y, n, seed, op, move="mala", eps=0.1)
    gpu = s.history(T + 1)[1:]
    assert [g["resampled"] for g in gpu] == [o.resampled for o in recs]
    assert abs(s.log_evidence() - ds_ref) < 1e-8
    assert abs(s.path_sampling() - ps_ref) < 1e-8


def test_adaptive_schedule_fp64_matches_oracle():
    """CESS-targeted tempering, FP64, free-running: the device's bisection
    picks the oracle's alpha_t at every iteration (the same float64
    midpoints and decisions), alpha reaches 1, and both evidence estimates
    match the oracle within 1e-8."""
    need_gpu()
    n, nd, r, T, seed = 2048, 100, 2, 40, 3
    s, y, op = make_gmm(n, nd=nd, r=r, T=T, precision=64, seed=seed, schedule="adaptive", ess_target=0.6)
    s.initialize()
    s.iterate(T)
    ds_ref, ps_ref, recs = ogmm.run(y, n, seed, op)
    gpu = s.history(T + 1)[1:]
    al_gpu = [g["alpha"] for g in gpu]
    al_ref = [o.alpha for o in recs]
    assert max(abs(a - b) for a, b in zip(al_gpu, al_ref)) < 1e-12, (al_gpu[:5], al_ref[:5])
    assert al_ref[-1] == 1.0 and 3 < sum(1 for a in al_ref if a < 1.0) < T
    assert [g["resampled"] for g in gpu] == [o.resampled for o in recs]
    assert abs(s.log_evidence() - ds_ref) < 1e-8
    assert abs(s.path_sampling() - ps_ref) < 1e-8


def test_adaptive_alpha_fp32_hits_the_cess_target():
    """FP32 at the benchmark's size: every alpha_t the device picks puts the
    conditional ESS of the GPU's own weights and log-likelihoods at the
    target (to float accuracy) unless it jumped to 1, and checkpoint resume
    continues the adaptive schedule bit for bit."""
    need_gpu()
    n, T, rho = 1 << 16, 40, 0.5
    s, y, op = make_gmm(n, nd=1000, r=4, T=T, precision=32, seed=5, schedule="adaptive", ess_target=rho)
    s.initialize()
    steps = 0
    blob = None
    for t in range(1, 13):
        x = s.state().astype(np.float64)
        lw = s.log_weight().astype(np.float64)
        prev = s.history(1)[0]
        logW = np.full(n, -math.log(n)) if prev["resampled"] else lw - prev["L"]
        llik = x[3 * 4 + 1]
        s.move()
        rec = s.history(1)[0]
        a_t, a_p = rec["alpha"], prev["alpha"]
        assert a_t > a_p or a_p == 1.0
        if a_t < 1.0:
            steps += 1
            lc = ogmm.log_cess(logW, llik, a_t - a_p)
            assert abs(lc - math.log(rho * n)) < 2e-4, (t, lc, math.log(rho * n))
        s.resample()
        s.mcmc()
        if t == 6:
            blob = s.checkpoint()
    assert steps >= 3
    s.iterate(5)
    ref = s.history(1)[0]
    b, _, _ = make_gmm(n, nd=1000, r=4, T=T, precision=32, seed=5, schedule="adaptive", ess_target=rho)
    b.restore(blob)
    b.iterate(6 + 5)
    got = b.history(1)[0]
    assert got["alpha"] == ref["alpha"] and got["logZ"] == ref["logZ"]


def test_langevin_benchmark_size_sampled():
    """The Langevin workload at its benchmarked size (N = 2^18, n = 1000,
    r = 4, step 0.05, FP32; 4096 blocks of mcmc partials, combined in
    several passes): sampled particles of a few iterations against the
    oracle's MALA step at their own slots, and their cached likelihood
    gradients against the oracle's."""
    need_gpu()
    n, r, seed, eps = 1 << 18, 4, 0, 0.05
    s, y, op = make_gmm(n, nd=1000, r=r, T=500, precision=32, seed=seed, move="mala", eps=eps)
    s.initialize()
    g = np.random.default_rng(9)
    idx = np.sort(g.choice(n, size=512, replace=False))
    near_total = 0
    for t in range(1, 4):
        s.move()
        rec = s.history(1)[0]
        s.resample()
        src = s.ancestors().astype(np.int64)[idx] if rec["resampled"] else idx
        xin = s.state().astype(np.float64)[:, src]
        mu, lam, om = xin[:r], xin[r:2 * r], xin[2 * r:3 * r]
        st = ogmm.State(mu.copy(), lam.copy(), om.copy(), ogmm.log_prior(mu, lam, om, op),
                        ogmm.log_lik(mu, lam, om, y))
        _, gm, gl, gz = ogmm.loglik_grad(st.mu, st.lam, st.om, y)
        ref = np.concatenate([gm, gl, gz])
        assert_close(xin[3 * r + 2:], ref, 2e-4 * np.max(np.abs(ref)), f"cached gradient t={t}")
        a_t = ogmm.alpha(t, op)
        ll_before = st.llik.copy()
        st, acc, delta, logu = ogmm.mala_step(st, a_t, t, y, seed, op, eps=eps, return_delta=True, slots=idx)
        near = np.abs(delta - logu) < _tie_window(32, a_t, ll_before, delta)
        near_total += int(near.sum())
        s.mcmc()
        x = s.state().astype(np.float64)[:, idx]
        ok = ~near
        assert_close(x[:r][:, ok], st.mu[:, ok], 1e-5, f"mu t={t}")
        assert_close(x[r:2 * r][:, ok], st.lam[:, ok], 1e-5, f"lambda t={t}")
        assert_close(x[2 * r:3 * r][:, ok], st.om[:, ok], 1e-5, f"omega t={t}")
        assert_close(x[3 * r + 1][ok], st.llik[ok], 1e-5, f"log-likelihood t={t}")
    assert near_total <= 0.01 * idx.size * 3 + 2
