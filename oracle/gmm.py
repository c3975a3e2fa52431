"""Bayesian Gaussian mixture model and its tempered SMC sampler.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 5.2 in float64:
* model (Sec. 5.2.1): y_k iid sum_j omega_j N(mu_j, 1 / lambda_j);
  priors mu_j ~ N(mu0, sd0^2), lambda_j ~ Gamma(shape0, rate0),
  omega ~ Dirichlet(1, ..., 1).  The log-prior keeps every normalising
  constant (the Dirichlet density on the simplex is Gamma(r)).
* log-likelihood l(theta) = sum_k log sum_j omega_j sqrt(lambda_j / 2 pi)
  exp(-lambda_j (y_k - mu_j)^2 / 2).  Reading: the paper sums the
  exponentials directly; here each datum uses a log-sum-exp over j (the
  same value, without underflow to -inf for far-off means).
* tempered targets gamma_t = prior * exp(alpha_t l) (eq:geometry) with
  alpha_t = t / T (linear) or (t / T)^p (prior), clamped to [0, 1]
  (Sec. 5.2.3, the alpha setter).
* Algorithm 2 for t = 1..T: incremental weights (alpha_t - alpha_{t-1}) l of
  the previous particles (eq:inc_weight_mcmc), normaliser, ESS test and
  resampling, then the pi_t-invariant kernel: three random-walk Metropolis
  blocks in this order (Sec. 5.2.1 list; the listing's mcmc queue order):
    mu:      mu' = mu + s_mu z;
    lambda:  log lambda' = log lambda + s_lam z, Jacobian sum log(lambda'/lambda);
    omega:   additive log-ratios z_j = log(omega_j / omega_r), j < r,
             z' = z + s_om eps, omega' = softmax([z', 0]), Jacobian
             sum_j log(omega'_j / omega_j).  Reading: the paper's "logit
             scale, that is, on omega_j/omega_r" is read as this transform.
  accept when log u <= Delta (the listing rejects when Delta < log u).
  Proposal scales from a = max(alpha_t, 0.02): s_mu = 0.15 / a,
  s_lam = (1 + sqrt(1 / a)) 0.15, s_om = (1 + sqrt(1 / a)) 0.2 (the move's
  hard-coded scales, Sec. 5.2.4).
* estimators: standard log Z = sum_t L_t (eq:smc-ds in the form of
  Algorithm 2: previous particles, normalised previous weights); path
  sampling sum_t (alpha_t - alpha_{t-1}) (U_t + U_{t-1}) / 2 with
  U_t = sum_i W_t,i l(theta_t,i) after the moves of iteration t and
  U_0 the mean log-likelihood of the prior draws (eq:path_est,
  eq:path_import; the integrand of eq:path_identity is l for this path).

Random numbers (Philox, counter index = particle slot):
* init (tag TAG_INIT, t = 0): mu from normals draws 0-1; lambda from
  shape0 exponentials per component, Exp number e = j * shape0 + m at word
  e % 4 of draw 8 + e // 4, divided by rate0; omega from r exponentials at
  draws 64-65, normalised.
* block b at iteration t (tags TAG_MH_MU / TAG_MH_LAMBDA / TAG_MH_WEIGHT):
  proposal normals from draws 0-1, acceptance uniform = word 0 of draw 16.

Parity pins (tests/test_oracle_gmm.py): l against enumeration over all
allocations for tiny n; log-prior against scipy.stats; for r = 1 the
evidence by one-dimensional quadrature (mu integrated out analytically)
against both estimators; T = 1 reduces to importance sampling from the
prior; at alpha = 0 the Metropolis blocks leave the prior invariant.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import philox, resample, weights

LOG_2PI = math.log(2.0 * math.pi)


@dataclass
class GMMParams:
    r: int = 4
    mu0: float = 0.0
    sd0: float = 10.0
    shape0: int = 1
    rate0: float = 1.0
    T: int = 500
    schedule: str = "prior"     # "linear", "prior" ((t/T)^power) or "adaptive" (CESS = ess_target N)
    power: float = 5.0
    ess_target: float = 0.5


def alpha(t, p):
    x = t / p.T
    a = x if p.schedule == "linear" else x ** p.power
    return min(max(a, 0.0), 1.0)


def log_prior(mu, lam, om, p):
    """mu, lam, om: (r, N).  Returns (N,)."""
    r = mu.shape[0]
    lp = np.sum(-0.5 * math.log(2 * math.pi * p.sd0 ** 2) - 0.5 * ((mu - p.mu0) / p.sd0) ** 2, axis=0)
    a, b = p.shape0, p.rate0
    with np.errstate(divide="ignore", invalid="ignore"):
        lp = lp + np.sum(a * math.log(b) - math.lgamma(a) + (a - 1) * np.log(lam) - b * lam, axis=0)
    lp = lp + math.lgamma(r)     # Dirichlet(1, ..., 1) on the simplex
    bad = np.any(lam <= 0, axis=0) | np.any(om < 0, axis=0)
    return np.where(bad, -np.inf, lp)


def log_lik(mu, lam, om, y, chunk=2048):
    """l(theta) for each particle; per-datum log-sum-exp over components."""
    r, N = mu.shape
    y = np.asarray(y, dtype=np.float64)
    out = np.empty(N)
    for s in range(0, N, chunk):
        m = mu[:, s:s + chunk, None]
        l_ = lam[:, s:s + chunk, None]
        w = om[:, s:s + chunk, None]
        with np.errstate(divide="ignore"):
            a = np.log(w) + 0.5 * np.log(l_) - 0.5 * LOG_2PI - 0.5 * l_ * (y[None, None, :] - m) ** 2
        amax = np.max(a, axis=0)
        ll = amax + np.log(np.sum(np.exp(a - amax[None]), axis=0))
        out[s:s + chunk] = np.sum(ll, axis=1)
    return out


@dataclass
class State:
    mu: np.ndarray
    lam: np.ndarray
    om: np.ndarray
    lprior: np.ndarray
    llik: np.ndarray

    def copy(self):
        return State(self.mu.copy(), self.lam.copy(), self.om.copy(), self.lprior.copy(), self.llik.copy())

    def take(self, idx):
        return State(self.mu[:, idx], self.lam[:, idx], self.om[:, idx], self.lprior[idx], self.llik[idx])


def init_state(n, y, seed, p, stream=0):
    idx = np.arange(n)
    z = philox.normals(seed, idx, 0, philox.TAG_INIT, p.r, stream)
    mu = p.mu0 + p.sd0 * z
    lam = np.zeros((p.r, n))
    for j in range(p.r):
        for m in range(p.shape0):
            e = j * p.shape0 + m
            w = philox.draw_words(seed, idx, 0, philox.TAG_INIT, stream, 8 + e // 4)
            lam[j] += -np.log(philox.uniform(w[:, e % 4]))
    lam /= p.rate0
    E = philox.exponentials(seed, idx, 0, philox.TAG_INIT, p.r, first_draw=64, stream=stream)
    om = E / np.sum(E, axis=0)
    return State(mu, lam, om, log_prior(mu, lam, om, p), log_lik(mu, lam, om, y))


def proposal_scales(a):
    a = max(a, 0.02)
    return 0.15 / a, (1 + math.sqrt(1 / a)) * 0.15, (1 + math.sqrt(1 / a)) * 0.2


def mh_block(s, block, a_t, t, y, seed, p, stream=0, return_delta=False, slots=None):
    """One Metropolis random-walk block at alpha_t.  Returns the new state
    and the acceptance indicators (and the log acceptance ratio and log u
    when asked).  slots: the particles' slots, i.e. their Philox counter
    indices (default 0 .. n-1; a subset of a larger system for sampled
    checks)."""
    n = s.mu.shape[1]
    idx = np.arange(n) if slots is None else np.asarray(slots)
    s_mu, s_lam, s_om = proposal_scales(a_t)
    tag = {"mu": philox.TAG_MH_MU, "lambda": philox.TAG_MH_LAMBDA, "weight": philox.TAG_MH_WEIGHT}[block]
    r = p.r
    mu, lam, om = s.mu.copy(), s.lam.copy(), s.om.copy()
    jac = np.zeros(n)
    if block == "mu":
        mu = mu + s_mu * philox.normals(seed, idx, t, tag, r, stream)
    elif block == "lambda":
        z = s_lam * philox.normals(seed, idx, t, tag, r, stream)
        lam = np.exp(np.log(lam) + z)
        jac = np.sum(z, axis=0)
    else:
        if r == 1:
            acc = np.ones(n, dtype=bool)
            return (s.copy(), acc, np.zeros(n), np.zeros(n)) if return_delta else (s.copy(), acc)
        zr = np.log(om[:-1] / om[-1:])
        zr = zr + s_om * philox.normals(seed, idx, t, tag, r - 1, stream)
        full = np.concatenate([zr, np.zeros((1, n))])
        full = full - np.max(full, axis=0)
        e = np.exp(full)
        om = e / np.sum(e, axis=0)
        jac = np.sum(np.log(om), axis=0) - np.sum(np.log(s.om), axis=0)
    lp = log_prior(mu, lam, om, p)
    ll = log_lik(mu, lam, om, y)
    delta = (lp + a_t * ll) - (s.lprior + a_t * s.llik) + jac
    w = philox.draw_words(seed, idx, t, tag, stream, philox.DRAW_MH_UNIFORM)
    logu = np.log(philox.uniform(w[:, 0]))
    acc = logu <= delta
    new = State(np.where(acc, mu, s.mu), np.where(acc, lam, s.lam), np.where(acc, om, s.om),
                np.where(acc, lp, s.lprior), np.where(acc, ll, s.llik))
    if return_delta:
        return new, acc, delta, logu
    return new, acc


def mcmc(s, a_t, t, y, seed, p, stream=0):
    accs = []
    for block in ("mu", "lambda", "weight"):
        s, acc = mh_block(s, block, a_t, t, y, seed, p, stream)
        accs.append(float(np.mean(acc)))
    return s, accs


@dataclass
class Iteration:
    t: int
    alpha: float
    lw: np.ndarray           # raw log-weights after the reweighting
    L: float                 # log-sum-exp = standard evidence increment
    ess: float
    resampled: bool
    ancestors: object
    state: State             # after the moves
    U: float                 # path-sampling integrand estimate U_t
    accept: list


def reweight(lw_prev, L_prev, resampled_prev, llik, a_prev, a_t):
    n = llik.shape[0]
    base = weights.previous_log_weight(lw_prev, L_prev, resampled_prev, n)
    lw = base + (a_t - a_prev) * llik
    _, L = weights.log_sum_exp(lw)
    return lw, L


# ---- adaptive tempering (Sec. 5.2.3 annealing schemes; ESS of Sec. 2.1) --
# Reading: the paper fixes alpha_t by a schedule; its adaptive variant here
# picks alpha_t so that the effective sample size of the incremental weights
# w_i = exp((alpha_t - alpha_{t-1}) l_i) under the current normalised weights
# W_{t-1,i}, the conditional ESS
#     CESS = N (sum_i W_i w_i)^2 / sum_i W_i w_i^2,
# equals rho N (CESS = N at alpha_t = alpha_{t-1}; the plain ESS of the
# product weights would already be below target when W_{t-1} is uneven).
# alpha_t = 1 when CESS at alpha = 1 is at least rho N; otherwise bisection on
# delta = alpha_t - alpha_{t-1} in [0, 1 - alpha_{t-1}] for a fixed number
# of halvings, keeping the lower end (CESS >= rho N there).

ADAPT_STEPS = 40


def log_cess(logW, llik, delta):
    """log CESS(delta) for normalised log-weights logW (float64)."""
    n = logW.shape[0]
    x = logW + delta * llik
    y = logW + 2.0 * delta * llik
    mx, my = float(np.max(x)), float(np.max(y))
    a = mx + math.log(float(np.sum(np.exp(x - mx))))
    b = my + math.log(float(np.sum(np.exp(y - my))))
    return math.log(n) + 2.0 * a - b


def adaptive_alpha(logW, llik, a_prev, rho, steps=ADAPT_STEPS):
    """alpha_t of the CESS-targeted schedule."""
    n = logW.shape[0]
    target = math.log(rho * n)
    hi = 1.0 - a_prev
    if hi <= 0.0:
        return 1.0
    if log_cess(logW, llik, hi) >= target:
        return 1.0
    lo = 0.0
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        if log_cess(logW, llik, mid) >= target:
            lo = mid
        else:
            hi = mid
    return min(1.0, a_prev + lo)


def path_u(lw, L, resampled, llik):
    n = llik.shape[0]
    if resampled:
        return float(np.mean(llik))
    return float(np.sum(np.exp(lw - L) * llik))


def run(y, n, seed, p, scheme="systematic", threshold=0.5, stream=0, keep=False, move="rw", eps=0.05):
    """Whole sampler.  Returns (log Z standard, log Z path sampling, records).
    move: "rw" (the three random-walk blocks), "mala" (one Langevin move) or
    "rw_mala" (the blocks, then one Langevin move).  With p.schedule
    "adaptive", alpha_t comes from adaptive_alpha with rho = p.ess_target and
    p.T is the most iterations run; iterations after alpha reaches 1 only
    move (their increment is zero)."""
    s = init_state(n, y, seed, p, stream)
    lw = np.full(n, -math.log(n))
    L = 0.0
    resampled = False
    a_prev = 0.0
    U_prev = float(np.mean(s.llik))
    logz_ds, logz_ps = 0.0, 0.0
    recs = []
    for t in range(1, p.T + 1):
        if p.schedule == "adaptive":
            logW = weights.previous_log_weight(lw, L, resampled, n)
            a_t = adaptive_alpha(logW, s.llik, a_prev, p.ess_target)
        else:
            a_t = alpha(t, p)
        lw, L = reweight(lw, L, resampled, s.llik, a_prev, a_t)
        W = np.exp(lw - L)
        e = 1.0 / float(np.sum(W * W))
        resampled = weights.resample_decision(e, n, threshold)
        anc = None
        if resampled:
            anc = resample.resample(scheme, lw, seed, t, stream)
            s = s.take(anc)
        accs = [0.0, 0.0, 0.0]
        if move in ("rw", "rw_mala"):
            s, accs = mcmc(s, a_t, t, y, seed, p, stream)
        if move in ("mala", "rw_mala"):
            s, am = mala_step(s, a_t, t, y, seed, p, eps, stream)
            accs = accs + [float(np.mean(am))]
        U = path_u(lw, L, resampled, s.llik)
        logz_ds += L
        logz_ps += 0.5 * (a_t - a_prev) * (U + U_prev)
        recs.append(Iteration(t, a_t, lw if keep else None, L, e, resampled, anc if keep else None,
                              s if keep else None, U, accs))
        U_prev, a_prev = U, a_t
    return logz_ds, logz_ps, recs


# ---------------------------------------------------------------- MALA --
# Not in the paper: the differentiable move asked of the hot path.  The
# Metropolis-adjusted Langevin move acts jointly on the unconstrained
# coordinates u = (mu_1..r, log lambda_1..r, z_1..r-1), z_j = log(omega_j /
# omega_r), targeting gamma_t(u) = log-prior + alpha_t l + log|Jacobian|
# (sum_j log lambda_j + sum_j log omega_j; the same Jacobians as the
# random-walk blocks).  With responsibilities rho_kj = omega_j N_kj / sum_i
# omega_i N_ki:
#   d gamma / d mu_j       = -(mu_j - mu0)/sd0^2 + alpha sum_k rho_kj lambda_j (y_k - mu_j)
#   d gamma / d log lam_j  = (shape0 - 1) - rate0 lambda_j + 1
#                            + alpha sum_k rho_kj (1 - lambda_j (y_k - mu_j)^2) / 2
#   d gamma / d z_j        = 1 - r omega_j + alpha sum_k (rho_kj - omega_j)
# Proposal u' = u + eps^2/2 grad(u) + eps xi; accept when
# log U <= gamma(u') - gamma(u) + log q(u | u') - log q(u' | u),
# log q(b | a) = -|b - a - eps^2/2 grad(a)|^2 / (2 eps^2).
# Random numbers: 3r - 1 normals from draws 0-2 of tag TAG_MALA, the
# acceptance uniform at draw 16.


def to_unconstrained(mu, lam, om):
    return np.concatenate([mu, np.log(lam), np.log(om[:-1] / om[-1:])])


def from_unconstrained(u, r):
    mu = u[:r]
    lam = np.exp(u[r:2 * r])
    full = np.concatenate([u[2 * r:], np.zeros((1, u.shape[1]))])
    full = full - np.max(full, axis=0)
    e = np.exp(full)
    return mu, lam, e / np.sum(e, axis=0)


def loglik_grad(mu, lam, om, y, chunk=1024):
    """l(theta) and its gradient in u: returns (l, d/dmu, d/dloglam, d/dz)."""
    r, N = mu.shape
    ll = np.empty(N)
    gmu = np.empty((r, N))
    glam = np.empty((r, N))
    gz = np.empty((max(r - 1, 0), N))
    for s in range(0, N, chunk):
        m = mu[:, s:s + chunk, None]
        l_ = lam[:, s:s + chunk, None]
        w = om[:, s:s + chunk, None]
        d = y[None, None, :] - m
        with np.errstate(divide="ignore"):
            a = np.log(w) + 0.5 * np.log(l_) - 0.5 * LOG_2PI - 0.5 * l_ * d * d
        amax = np.max(a, axis=0)
        e = np.exp(a - amax[None])
        se = np.sum(e, axis=0)
        ll[s:s + chunk] = np.sum(amax + np.log(se), axis=1)
        rho = e / se[None]
        gmu[:, s:s + chunk] = np.sum(rho * l_ * d, axis=2)
        glam[:, s:s + chunk] = np.sum(rho * 0.5 * (1 - l_ * d * d), axis=2)
        if r > 1:
            gz[:, s:s + chunk] = np.sum(rho[:-1] - w[:-1], axis=2)
    return ll, gmu, glam, gz


def log_target_u(u, a_t, y, p):
    mu, lam, om = from_unconstrained(u, p.r)
    with np.errstate(divide="ignore"):
        jac = np.sum(np.log(lam), axis=0) + np.sum(np.log(om), axis=0)
    return log_prior(mu, lam, om, p) + a_t * log_lik(mu, lam, om, y) + jac


def grad_log_target_u(u, a_t, y, p):
    r = p.r
    mu, lam, om = from_unconstrained(u, r)
    ll, gmu, glam, gz = loglik_grad(mu, lam, om, y)
    g_mu = -(mu - p.mu0) / p.sd0 ** 2 + a_t * gmu
    g_lam = (p.shape0 - 1) - p.rate0 * lam + 1 + a_t * glam
    g_z = (1 - r * om[:-1]) + a_t * gz
    return np.concatenate([g_mu, g_lam, g_z]), ll


def mala_step(s, a_t, t, y, seed, p, eps=0.05, stream=0, return_delta=False, slots=None):
    """One Langevin (MALA) move at alpha_t in the unconstrained coordinates;
    slots as in mh_block."""
    n = s.mu.shape[1]
    r = p.r
    idx = np.arange(n) if slots is None else np.asarray(slots)
    u = to_unconstrained(s.mu, s.lam, s.om)
    g, _ = grad_log_target_u(u, a_t, y, p)
    xi = philox.normals(seed, idx, t, philox.TAG_MALA, 3 * r - 1, stream)
    up = u + 0.5 * eps * eps * g + eps * xi
    gp, llp = grad_log_target_u(up, a_t, y, p)
    mu, lam, om = from_unconstrained(up, r)
    lp = log_prior(mu, lam, om, p)
    with np.errstate(divide="ignore"):
        gam_p = lp + a_t * llp + np.sum(np.log(lam), axis=0) + np.sum(np.log(om), axis=0)
        gam = s.lprior + a_t * s.llik + np.sum(np.log(s.lam), axis=0) + np.sum(np.log(s.om), axis=0)
    fwd = -np.sum((up - u - 0.5 * eps * eps * g) ** 2, axis=0) / (2 * eps * eps)
    bwd = -np.sum((u - up - 0.5 * eps * eps * gp) ** 2, axis=0) / (2 * eps * eps)
    delta = gam_p - gam + bwd - fwd
    w = philox.draw_words(seed, idx, t, philox.TAG_MALA, stream, philox.DRAW_MH_UNIFORM)
    logu = np.log(philox.uniform(w[:, 0]))
    acc = logu <= delta
    new = State(np.where(acc, mu, s.mu), np.where(acc, lam, s.lam), np.where(acc, om, s.om),
                np.where(acc, lp, s.lprior), np.where(acc, llp, s.llik))
    if return_delta:
        return new, acc, delta, logu
    return new, acc
