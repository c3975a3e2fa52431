"""Almost-constant-velocity tracking model and its bootstrap particle filter.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 5.1.1 (the model and Algorithm 1) in float64:
* state X_t = (x_pos, y_pos, x_vel, y_vel); X_t = A X_{t-1} + V_t with
  independent normal noise, sd sigma_pos on positions and sigma_vel on
  velocities; positions move by Delta times the previous velocity.
  Reading: the printed matrix A is garbled (Delta sits in the position-
  position block); the listed move step adds Delta * velocity to the matching
  position, which is the reading used here:
  A = [[1,0,D,0],[0,1,0,D],[0,0,1,0],[0,0,0,1]].
* observation Y_t = (x_pos, y_pos) + scale * W_t, W_t iid Student-t with
  nu degrees of freedom.  Reading: the paper's log-likelihood drops the
  Student-t normalising constant; the full density is used here, so the
  estimate is a true log-likelihood.  The Gaussian variant replaces W_t by
  standard normals (closed form via the Kalman filter, ``oracle.kalman``).
* prior X_0 ~ N(0, diag(sd_pos0^2, sd_pos0^2, sd_vel0^2, sd_vel0^2)),
  weighted by the likelihood of Y_0, then one move + weight per later datum
  (Algorithm 1; the listing's main function initialises on datum 0 and
  iterates DataNum - 1 times).
* after every weighting: ESS test, then resampling (``oracle.resample``);
  the gather x'_k = x_{a_k} happens at the start of the next move
  (Sec. 4.1.2, copy_from).
* monitor: the filtered mean sum_i W_t,i pos_i of the two positions, taken
  after weighting and before resampling (reading: vSMC records monitors after
  the whole iteration; the pre-resampling estimate is the lower-variance one).
  The post-resampling mean (Sec. 4.1.5 evaluates monitors after the whole
  iteration) is also reported: (1/N) sum_k pos_{a_k} over the resampled
  system when the iteration resampled, else the weighted mean itself (the
  particle system after the iteration is then the weighted one).
* the log-likelihood estimate log Z-hat = sum_t L_t, L_t the log-sum-exp of
  lw_t = log W_{t-1} + log g(y_t | x_t) (Sec. 2.2 ratio estimator).

Random numbers: four normals per particle per iteration from Philox with
tag TAG_MOVE (TAG_INIT at t = 0), counter index = particle slot, mapped to
(x_pos, y_pos, x_vel, y_vel) noise in that order.

Parity pins: Student-t density against scipy.stats.t (test_oracle_cv);
the Gaussian variant's evidence estimate against the Kalman-filter closed
form over many seeds; zero-noise moves reduce to multiplication by A.
"""
import math
from dataclasses import dataclass

import numpy as np

from . import philox, resample, weights


@dataclass
class CVParams:
    delta: float = 0.1
    sd_pos: float = 0.02
    sd_vel: float = 1.0
    obs_scale: float = 0.5
    obs_df: float = 10.0
    sd_pos0: float = 1.0
    sd_vel0: float = 1.0
    gaussian_obs: bool = False


def transition_matrix(delta):
    return np.array([[1, 0, delta, 0], [0, 1, 0, delta], [0, 0, 1, 0], [0, 0, 0, 1]],
                    dtype=np.float64)


def student_t_const(p):
    nu, s = p.obs_df, p.obs_scale
    return (math.lgamma((nu + 1) / 2) - math.lgamma(nu / 2)
            - 0.5 * math.log(nu * math.pi) - math.log(s))


def loglik(x, y_t, p):
    """log g(y_t | x) for each particle; x is (4, n)."""
    zx = (y_t[0] - x[0]) / p.obs_scale
    zy = (y_t[1] - x[1]) / p.obs_scale
    if p.gaussian_obs:
        c = -0.5 * math.log(2 * math.pi) - math.log(p.obs_scale)
        return 2 * c - 0.5 * (zx * zx + zy * zy)
    nu = p.obs_df
    c = student_t_const(p)
    return (2 * c - 0.5 * (nu + 1) * (np.log1p(zx * zx / nu) + np.log1p(zy * zy / nu)))


def init_state(n, seed, p, stream=0, index=None):
    """Prior draws of particles `index` (default 0 .. n-1; a sub-range lets
    the particles be drawn in independent blocks)."""
    idx = np.arange(n) if index is None else np.asarray(index)
    eps = philox.normals(seed, idx, 0, philox.TAG_INIT, 4, stream)
    return np.stack([eps[0] * p.sd_pos0, eps[1] * p.sd_pos0,
                     eps[2] * p.sd_vel0, eps[3] * p.sd_vel0])


def move(x, t, seed, p, stream=0, index=None):
    """One draw of X_t = A X_{t-1} + V_t per particle (Algorithm 1); the
    columns of x are the particles `index` (default 0 .. n-1)."""
    n = x.shape[1]
    idx = np.arange(n) if index is None else np.asarray(index)
    eps = philox.normals(seed, idx, t, philox.TAG_MOVE, 4, stream)
    return np.stack([x[0] + p.delta * x[2] + p.sd_pos * eps[0],
                     x[1] + p.delta * x[3] + p.sd_pos * eps[1],
                     x[2] + p.sd_vel * eps[2],
                     x[3] + p.sd_vel * eps[3]])


@dataclass
class StepResult:
    x: np.ndarray          # (4, n) state after the move
    lw: np.ndarray         # raw log-weights lw_t
    L: float               # log-sum-exp of lw_t = log Z_t / Z_{t-1}
    ess: float
    mean_x: float
    mean_y: float
    resample: bool         # ESS test outcome


def weigh(x, base, y_t, p, threshold):
    lw = base + loglik(x, y_t, p)
    _, L = weights.log_sum_exp(lw)
    W = np.exp(lw - L)
    e = 1.0 / float(np.sum(W * W))
    n = x.shape[1]
    return StepResult(x, lw, L, e, float(np.sum(W * x[0])), float(np.sum(W * x[1])),
                      weights.resample_decision(e, n, threshold))


def init_step(n, y0, seed, p, threshold, stream=0):
    x = init_state(n, seed, p, stream)
    return weigh(x, np.full(n, -math.log(n)), y0, p, threshold)


def step(x_prev, lw_prev, L_prev, ancestors, t, y_t, seed, p, threshold, stream=0):
    """Iteration t >= 1: gather (if the previous iteration resampled, i.e.
    ``ancestors`` is not None), move, weight, normalise, ESS test."""
    n = x_prev.shape[1]
    if ancestors is not None:
        x_prev = x_prev[:, np.asarray(ancestors, dtype=np.int64)]
        base = np.full(n, -math.log(n))
    else:
        base = np.asarray(lw_prev, dtype=np.float64) - L_prev
    return weigh(move(x_prev, t, seed, p, stream), base, y_t, p, threshold)


def post_resampling_mean(r, ancestors):
    """Mean of the two positions over the particle system that ends the
    iteration: equally weighted copies x_{a_k} after resampling, else the
    weighted system (its weighted mean)."""
    if ancestors is None:
        return r.mean_x, r.mean_y
    a = np.asarray(ancestors, dtype=np.int64)
    return float(np.mean(r.x[0][a])), float(np.mean(r.x[1][a]))


def run(y, n, seed, p, scheme="systematic", threshold=0.5, stream=0, record_ancestors=False, inplace=False):
    """Whole filter over observations y (T, 2).  Returns per-iteration
    records and the final state.  inplace: each step's ancestors in the
    in-place copy_from arrangement (``resample.stay_permutation``)."""
    T = y.shape[0]
    recs = []
    r = init_step(n, y[0], seed, p, threshold, stream)
    anc = None
    logZ = 0.0
    for t in range(T):
        if t > 0:
            r = step(r_prev.x, r_prev.lw, r_prev.L, anc, t, y[t], seed, p, threshold, stream)
        logZ += r.L
        anc = resample.resample(scheme, r.lw, seed, t, stream) if r.resample else None
        if inplace and anc is not None:
            anc = resample.stay_permutation(anc)
        post = post_resampling_mean(r, anc)
        rec = dict(t=t, L=r.L, logZ=logZ, ess=r.ess, mean_x=r.mean_x, mean_y=r.mean_y,
                   resampled=r.resample, post_mean_x=post[0], post_mean_y=post[1])
        if record_ancestors:
            rec["ancestors"] = anc
        recs.append(rec)
        r_prev = r
    return recs, r
