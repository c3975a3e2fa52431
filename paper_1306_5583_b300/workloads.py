"""Seeded synthetic inputs for the SMC workloads.

This module only draws data; it holds none of the filter's or sampler's
arithmetic.  It uses numpy's PCG64 generator (not the method's Philox
streams), so the data are independent of every draw the method makes.

* ``cv_data``: a trajectory and its observations from the almost-constant-
  velocity model of Sec. 5.1.1 (x_0 ~ N(0, diag(sd_pos0^2, sd_pos0^2,
  sd_vel0^2, sd_vel0^2)); x_t = A x_{t-1} + normal noise; y_t = position +
  scale * Student-t(nu) noise, or normal noise for the Gaussian variant).
  Stands in for the paper's missing data file of 100 observations.
* ``gmm_data``: n points from an equal-weight normal mixture (Sec. 5.2.1:
  means (-3, 0, 3, 6); unit variance for the default workload).
* ``batch_shapes``: per-filter particle counts (log-uniform in
  [2^10, 2^18]) and lengths (uniform in [50, 2000]) of the batched workload.
"""
import numpy as np

# default model constants of the benchmarked workloads
CV_DEFAULT = dict(delta=0.1, sd_pos=0.02, sd_vel=1.0, obs_scale=0.5, obs_df=10.0,
                  sd_pos0=1.0, sd_vel0=1.0)
# the constants printed in Sec. 5.1.1 (variances 0.02 / 0.001, prior
# variances 4 / 1, observation scale 0.1)
CV_PAPER = dict(delta=0.1, sd_pos=0.02 ** 0.5, sd_vel=0.001 ** 0.5, obs_scale=0.1,
                obs_df=10.0, sd_pos0=2.0, sd_vel0=1.0)


def cv_data(T, seed=0, delta=0.1, sd_pos=0.02, sd_vel=1.0, obs_scale=0.5, obs_df=10.0,
            sd_pos0=1.0, sd_vel0=1.0, gaussian_obs=False):
    """Returns (x, y): true states (T, 4) and observations (T, 2), float64."""
    g = np.random.default_rng(seed)
    x = np.empty((T, 4))
    y = np.empty((T, 2))
    s0 = np.array([sd_pos0, sd_pos0, sd_vel0, sd_vel0])
    sq = np.array([sd_pos, sd_pos, sd_vel, sd_vel])
    cur = g.standard_normal(4) * s0
    for t in range(T):
        if t > 0:
            nxt = cur.copy()
            nxt[0] = cur[0] + delta * cur[2]
            nxt[1] = cur[1] + delta * cur[3]
            cur = nxt + g.standard_normal(4) * sq
        x[t] = cur
        noise = g.standard_normal(2) if gaussian_obs else g.standard_t(obs_df, size=2)
        y[t] = cur[:2] + obs_scale * noise
    return x, y


def gmm_data(n=1000, seed=0, means=(-3.0, 0.0, 3.0, 6.0), sd=1.0):
    """n iid draws from the equal-weight mixture sum_j N(means_j, sd^2)/r."""
    g = np.random.default_rng(seed)
    comp = g.integers(0, len(means), size=n)
    return np.asarray(means)[comp] + sd * g.standard_normal(n)


def batch_shapes(count=256, seed=0, log2_lo=10, log2_hi=18, t_lo=50, t_hi=2000):
    """(N_b, T_b) of `count` filters: N_b = round(exp(U(ln 2^lo, ln 2^hi))),
    T_b uniform on {t_lo, ..., t_hi}."""
    g = np.random.default_rng(seed)
    n = np.rint(np.exp(g.uniform(log2_lo * np.log(2), log2_hi * np.log(2), size=count)))
    t = g.integers(t_lo, t_hi + 1, size=count)
    return n.astype(np.int64), t.astype(np.int64)
