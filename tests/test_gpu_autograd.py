"""torch.autograd.Function wrappers over the hand-written adjoints: the GMM
tempered log-target (values and gradients against the oracle's analytic FP64
gradient) and the particle filter's log-likelihood estimate (the backward
pass is the reverse sweep of smc_pf_grad)."""
import numpy as np
import pytest

from gpu_common import assert_close, make_pf, need_gpu, torch
from oracle import gmm as ogmm
from paper_1306_5583_b300 import autograd, smc, workloads

pytestmark = pytest.mark.gpu


def _points(count, r, seed):
    g = np.random.default_rng(seed)
    mu = g.normal(scale=3, size=(r, count))
    lam = g.gamma(2.0, 1.0, size=(r, count))
    om = g.dirichlet(np.ones(r), size=count).T
    return ogmm.to_unconstrained(mu, lam, om)


@pytest.mark.parametrize("precision,rel", [(64, 1e-10), (32, 2e-5)])
def test_gmm_log_target_and_gradient_match_oracle(precision, rel):
    need_gpu()
    r, nd, count = 4, 250, 700
    y = workloads.gmm_data(nd, seed=3)
    cfg = smc.make_config(model="gmm", n=1024, precision=precision, max_data=nd, max_records=8,
                          gmm=dict(n_comp=r, n_iter=5, move=smc.GMM_MALA, mala_step=0.05))
    s = smc.Sampler(cfg)
    s.set_data(y)
    op = ogmm.GMMParams(r=r)
    u = _points(count, r, 1)
    dt = torch.float64 if precision == 64 else torch.float32
    for alpha in (0.0, 0.37, 1.0):
        ut = torch.tensor(u.T, dtype=dt, device="cuda", requires_grad=True)
        val = autograd.GMMLogTarget.apply(ut, s, alpha)
        (g,) = torch.autograd.grad(val.sum(), ut)
        ref_v = ogmm.log_target_u(u, alpha, y.astype(np.float64) if precision == 64 else y.astype(np.float32)
                                  .astype(np.float64), op)
        ref_g, _ = ogmm.grad_log_target_u(u, alpha, y.astype(np.float64) if precision == 64 else
                                          y.astype(np.float32).astype(np.float64), op)
        assert_close(val.detach().cpu().numpy(), ref_v, rel, f"log-target alpha={alpha}")
        assert_close(g.cpu().numpy().T, ref_g, 20 * rel, f"gradient alpha={alpha}")


def test_pf_log_likelihood_autograd_is_the_reverse_sweep():
    need_gpu()
    T, n, seed = 25, 4096, 3
    p = dict(workloads.CV_DEFAULT)
    _, y = workloads.cv_data(T, seed=1, **p)
    theta = torch.tensor([p["sd_pos"], p["sd_vel"], p["obs_scale"], p["obs_df"]], dtype=torch.float64,
                         requires_grad=True)
    out = autograd.PFLogLikelihood.apply(theta, y, n, seed, 64)
    out.backward()
    # the same recorded run through the sampler API
    cfg = smc.make_config(model="cv", n=n, precision=64, seed=seed, max_data=T, max_records=T, cv=p,
                          keep_cdf=False, record=True)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(T - 1)
    assert out.item() == s.log_evidence()
    assert np.array_equal(theta.grad.numpy(), s.pf_grad())
    # and a central difference of the replayed estimate agrees
    h = 1e-4
    for j in range(4):
        tp = theta.detach().numpy().copy()
        tm = tp.copy()
        tp[j] += h * tp[j]
        tm[j] -= h * tm[j]
        fd = (s.pf_replay(tp) - s.pf_replay(tm)) / (tp[j] - tm[j])
        assert abs(theta.grad[j].item() - fd) <= 1e-5 * max(abs(fd), 1.0), (j, theta.grad[j].item(), fd)
