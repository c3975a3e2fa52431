"""Gradient of the particle filter's log-likelihood estimate.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper: the differentiable form asked of the hot path.  The
estimate log Z-hat = sum_t L_t of ``oracle.cv`` (Sec. 5.1, Algorithm 1;
Sec. 2.2 ratio estimator) is differentiated with respect to
theta = (sd_pos, sd_vel, obs_scale, obs_df) with the resampling held fixed
(stop-gradient resampling): the ancestors and the resampling decisions of a
base run are replayed, and the noise is reparameterised,
X_t = A X_{t-1, parent} + diag(sd_pos, sd_pos, sd_vel, sd_vel) eps_t with eps_t
fixed by the Philox counters.

Reverse mode, t = T-1 down to 0 (all float64):
* gbar_t = dJ/dlw_t: W_t, plus gbar_{t+1} - W_t sum(gbar_{t+1}) when
  iteration t did not resample (then lw_{t+1} = lw_t - L_t + log g);
* xbar_t = (adjoint from the children at t+1 through A^T) + gbar_t dlog g/dx;
* dJ/d(s, nu) += sum_i gbar_t,i dlog g_t,i/d(s, nu); dJ/d(sd_pos, sd_vel)
  += sum_i xbar_t,i . d x_t,i / d sd (the eps of the move);
* parents at t-1 collect A^T xbar_t of their children.

Student-t observation term per coordinate, z = (y - x)/s:
  dlog g/dx = (nu + 1) z / (s (nu + z^2)),
  dlog g/ds = -1/s + (nu + 1) z^2 / (s (nu + z^2)),
  dlog g/dnu = (psi((nu + 1)/2) - psi(nu/2)) / 2 - 1/(2 nu)
               - log(1 + z^2/nu) / 2 + (nu + 1) z^2 / (2 nu (nu + z^2)).
Gaussian variant: dlog g/dx = z/s, dlog g/ds = -1/s + z^2/s.

Parity pin (tests/test_oracle_grad.py): central finite differences of the
replayed estimate (h = 1e-3 relative) for every component.
"""
import math

import numpy as np
from scipy.special import digamma

from . import cv, philox, weights

THETA = ("sd_pos", "sd_vel", "obs_scale", "obs_df")


def with_theta(p, theta):
    return cv.CVParams(delta=p.delta, sd_pos=theta[0], sd_vel=theta[1], obs_scale=theta[2], obs_df=theta[3],
                       sd_pos0=p.sd_pos0, sd_vel0=p.sd_vel0, gaussian_obs=p.gaussian_obs)


def base_run(y, n, seed, p, scheme="systematic", threshold=0.5):
    """Forward run recording the resampling (decisions and ancestors)."""
    recs, _ = cv.run(y, n, seed, p, scheme=scheme, threshold=threshold, record_ancestors=True)
    return [r["ancestors"] for r in recs]


def replay(y, n, seed, p, ancestors):
    """Forward pass with the recorded resampling; returns log Z-hat and the
    per-iteration particle systems (x_t, lw_t, L_t)."""
    T = y.shape[0]
    xs, lws, Ls = [], [], []
    x = cv.init_state(n, seed, p)
    lw = np.full(n, -math.log(n)) + cv.loglik(x, y[0], p)
    for t in range(T):
        if t > 0:
            prev_anc = ancestors[t - 1]
            if prev_anc is not None:
                xp = x[:, prev_anc]
                base = np.full(n, -math.log(n))
            else:
                xp = x
                base = lw - Ls[-1]
            x = cv.move(xp, t, seed, p)
            lw = base + cv.loglik(x, y[t], p)
        _, L = weights.log_sum_exp(lw)
        xs.append(x)
        lws.append(lw)
        Ls.append(L)
    return float(sum(Ls)), xs, lws, Ls


def dloglik(x, y_t, p):
    """(d/dx_pos, d/dy_pos, d/ds, d/dnu) of log g(y_t | x) per particle."""
    s, nu = p.obs_scale, p.obs_df
    zx = (y_t[0] - x[0]) / s
    zy = (y_t[1] - x[1]) / s
    if p.gaussian_obs:
        return zx / s, zy / s, (-1 / s + zx * zx / s) + (-1 / s + zy * zy / s), np.zeros_like(zx)
    gx = (nu + 1) * zx / (s * (nu + zx * zx))
    gy = (nu + 1) * zy / (s * (nu + zy * zy))
    ds = sum(-1 / s + (nu + 1) * z * z / (s * (nu + z * z)) for z in (zx, zy))
    c = 0.5 * (digamma((nu + 1) / 2) - digamma(nu / 2)) - 0.5 / nu
    dnu = sum(c - 0.5 * np.log1p(z * z / nu) + (nu + 1) * z * z / (2 * nu * (nu + z * z)) for z in (zx, zy))
    return gx, gy, ds, dnu


def gradient(y, n, seed, p, ancestors):
    """Reverse-mode gradient of the replayed log Z-hat."""
    T = y.shape[0]
    J, xs, lws, Ls = replay(y, n, seed, p, ancestors)
    g = np.zeros(4)
    xbar_next = np.zeros((4, n))
    gbar_next = None
    for t in range(T - 1, -1, -1):
        W = np.exp(lws[t] - Ls[t])
        if t == T - 1 or ancestors[t] is not None:
            gbar = W
        else:
            gbar = W + gbar_next - W * np.sum(gbar_next)
        gx, gy, ds, dnu = dloglik(xs[t], y[t], p)
        xbar = xbar_next.copy()
        xbar[0] += gbar * gx
        xbar[1] += gbar * gy
        g[2] += np.sum(gbar * ds)
        g[3] += np.sum(gbar * dnu)
        if t > 0:
            eps = philox.normals(seed, np.arange(n), t, philox.TAG_MOVE, 4)
            g[0] += np.sum(xbar[0] * eps[0] + xbar[1] * eps[1])
            g[1] += np.sum(xbar[2] * eps[2] + xbar[3] * eps[3])
            # A^T xbar: positions pass through, velocities collect delta * position adjoint
            at = np.stack([xbar[0], xbar[1], xbar[2] + p.delta * xbar[0], xbar[3] + p.delta * xbar[1]])
            anc = ancestors[t - 1]
            if anc is None:
                xbar_next = at
            else:
                xbar_next = np.zeros((4, n))
                for r in range(4):
                    np.add.at(xbar_next[r], anc, at[r])
        gbar_next = gbar
    return J, g


def finite_difference(y, n, seed, p, ancestors, h=1e-3):
    """Central differences of the replayed estimate, step h * theta_j."""
    theta = [getattr(p, k) for k in THETA]
    out = np.zeros(4)
    for j in range(4):
        tp = list(theta)
        tm = list(theta)
        tp[j] += h * theta[j]
        tm[j] -= h * theta[j]
        jp = replay(y, n, seed, with_theta(p, tp), ancestors)[0]
        jm = replay(y, n, seed, with_theta(p, tm), ancestors)[0]
        out[j] = (jp - jm) / (2 * h * theta[j])
    return out
