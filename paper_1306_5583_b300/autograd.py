"""torch.autograd.Function wrappers over the library's hand-written adjoints.

* GMMLogTarget: per-point tempered log-target gamma_alpha(u) of the
  Gaussian-mixture model (Sec. 5.2) in unconstrained coordinates; backward
  uses the gradient that the same kernel computes (smc_gmm_log_target).
* PFLogLikelihood: the particle filter's log-likelihood estimate log Z-hat
  (Sec. 5.1, Algorithm 1) as a function of theta = (sd_pos, sd_vel,
  obs_scale, obs_df); backward is the reverse sweep with the resampling of
  the forward run held fixed (smc_pf_grad).

Marshalling only: every value and gradient comes from the CUDA kernels.
"""
import numpy as np
import torch

from . import smc


class GMMLogTarget(torch.autograd.Function):
    """gamma = GMMLogTarget.apply(u, sampler, alpha): u (count, 3r - 1)."""

    @staticmethod
    def forward(ctx, u, sampler, alpha):
        logt, grad = sampler.gmm_log_target(u, alpha)
        ctx.save_for_backward(grad)
        return logt.to(u.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g.to(grad.dtype)[:, None] * grad).to(g.dtype), None, None


THETA = ("sd_pos", "sd_vel", "obs_scale", "obs_df")


def _pf_sampler(theta, y, n, seed, precision, scheme, threshold, model, base):
    p = dict(base)
    for k, v in zip(THETA, theta):
        p[k] = float(v)
    T = y.shape[0]
    cfg = smc.make_config(model=model, n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=T, max_records=T, cv=p, keep_cdf=False, record=True)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    s.iterate(T - 1)
    return s


class PFLogLikelihood(torch.autograd.Function):
    """logZ = PFLogLikelihood.apply(theta, y, n, seed, precision, scheme,
    threshold, model, base): theta a 4-vector tensor, y (T, 2) observations,
    base the other CV parameters (workloads.CV_DEFAULT keys)."""

    @staticmethod
    def forward(ctx, theta, y, n, seed, precision=32, scheme="systematic", threshold=0.5, model="cv", base=None):
        from . import workloads
        b = dict(workloads.CV_DEFAULT if base is None else base)
        th = theta.detach().cpu().double().numpy()
        s = _pf_sampler(th, np.asarray(y, dtype=np.float64), int(n), int(seed), precision, scheme, threshold, model,
                        b)
        ctx.sampler = s
        return torch.tensor(s.log_evidence(), dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        grad = torch.tensor(ctx.sampler.pf_grad(), dtype=g.dtype, device=g.device)
        ctx.sampler.close()
        return (g * grad,) + (None,) * 8
