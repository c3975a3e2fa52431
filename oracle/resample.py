"""Resampling: fixed-point CDF and the four ancestor-selection schemes.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.1 (eq:resample and the paragraph after it): resampling draws integer
replication counts R_i >= 0 with sum N such that the resampled system has the
same expectation; the multinomial distribution with the normalised weights is
one such law, and Douc et al. (2005) list the commonly used alternatives
(stratified, systematic, residual).  Sec. 4.1.2 fixes the output convention:
copy_from[k] is the parent of new particle k.

Readings (the paper is silent on the arithmetic; the same readings bind the
CUDA path):
* Fixed-point weights.  With m = max lw and F = 61 - ceil(log2 N) fraction
  bits, q_i = floor(exp(lw_i - m) * 2^F) and Q_i = q_0 + ... + q_i are exact
  integers (Q_N <= N 2^F <= 2^61).  Resampling is exact, order-independent
  and deterministic in this representation; a particle whose weight is below
  2^-F of the largest one gets weight zero.
* Targets are rationals P_k / D with D = N 2^25 and the uniform
  u = (2j + 1) / 2^25 of ``oracle.philox``:
    systematic  P_k = 2^25 k + 2j + 1, one j per iteration;
    stratified  P_k = 2^25 k + 2j_k + 1, j_k independent;
    multinomial P_k = N (2 j_(k) + 1), j_(k) the k-th smallest of N iid j's
                (sorting the iid uniforms does not change the multiset of
                ancestors, and the ancestor multiset defines the scheme).
* Selection: a_k = min{ i : Q_i D > Q_N P_k } (an upper bound).  Particles
  with q_i = 0 are never selected.  The ancestors come out sorted.
* Residual (multinomial residual step): d_i = floor(N q_i / Q_N) copies,
  rem_i = N q_i - d_i Q_N, R = N - sum d_i residual draws; the residual
  weights are r_i = rem_i >> s with s = max(0, bitlength(R Q_N) - 62)
  (sum rem_i = R Q_N exactly, so the residual CDF fits in 62 bits and is
  nonzero whenever R > 0); the R residual ancestors come from multinomial
  selection on the r-CDF with R sorted iid uniforms; the final ancestors are
  the sorted expansion of the counts d_i + (residual draws of i).

Residual variants (Douc et al. 2005): the R residual outputs drawn by
systematic (one uniform) or stratified (one uniform per output) selection on
the residual CDF instead of multinomially, targets P_k / D with D = R 2^25.

Parity pins (tests/test_oracle_resample.py): sum of counts = N; exact
unbiasedness E[o_i] = N q_i / Q_N by enumeration of all 2^24 systematic
uniforms for tiny N; Monte Carlo unbiasedness (5 sigma) for stratified,
multinomial and residual; systematic counts within {floor, ceil} of N W_i;
residual counts >= floor(N W_i); sorted output; zero-weight particles never
selected.
"""
import math

import numpy as np

from . import philox


def frac_bits(n):
    """F = 61 - ceil(log2 N)."""
    return 61 - max(0, (int(n) - 1).bit_length())


def quantise(lw):
    """q_i = floor(exp(lw_i - m) 2^F) as Python ints (object array)."""
    lw = np.asarray(lw, dtype=np.float64)
    n = lw.shape[0]
    m = float(np.max(lw))
    if not math.isfinite(m):
        raise FloatingPointError("all log-weights are -inf or NaN")
    scale = 2.0 ** frac_bits(n)
    e = np.exp(lw - m)
    return np.array([int(math.floor(v * scale)) for v in e], dtype=object)


def cdf(q):
    """Inclusive prefix sums Q_i of the fixed-point weights (exact)."""
    out = np.empty(len(q), dtype=object)
    acc = 0
    for i, v in enumerate(q):
        acc += int(v)
        out[i] = acc
    return out


def select(Q, P, D):
    """a_k = min{i : Q_i D > Q_N P_k}, for non-decreasing numerators P."""
    Q = [int(v) for v in Q]
    QN = Q[-1]
    if QN <= 0:
        raise FloatingPointError("total fixed-point weight is zero")
    # Q_i D > Q_N P_k  <=>  Q_i > floor(Q_N P_k / D)   (Q_i integer)
    thr = [(QN * int(p)) // int(D) for p in P]
    import bisect
    return np.array([bisect.bisect_right(Q, t) for t in thr], dtype=np.int64)


def systematic_targets(n, j):
    return [(k << 25) + 2 * int(j) + 1 for k in range(n)], n << 25


def stratified_targets(n, js):
    return [(k << 25) + 2 * int(js[k]) + 1 for k in range(n)], n << 25


def multinomial_targets(n, js):
    s = sorted(int(v) for v in js)
    return [n * (2 * v + 1) for v in s], n << 25


def systematic(Q, seed, t, stream=0):
    n = len(Q)
    P, D = systematic_targets(n, philox.systematic_u24(seed, t, stream))
    return select(Q, P, D)


def stratified(Q, seed, t, stream=0):
    n = len(Q)
    P, D = stratified_targets(n, philox.resample_u24(seed, t, n, stream))
    return select(Q, P, D)


def multinomial(Q, seed, t, stream=0):
    n = len(Q)
    P, D = multinomial_targets(n, philox.resample_u24(seed, t, n, stream))
    return select(Q, P, D)


def residual_parts(q):
    """Deterministic copies d_i, residual draw count R, residual weights r_i
    and the shift s (see the module docstring)."""
    q = [int(v) for v in q]
    n = len(q)
    QN = sum(q)
    d = [(n * v) // QN for v in q]
    rem = [n * v - di * QN for v, di in zip(q, d)]
    R = n - sum(d)
    s = max(0, (R * QN).bit_length() - 62)
    r = [v >> s for v in rem]
    return d, R, r, s


def residual(q, seed, t, stream=0, step="multinomial"):
    """Residual resampling from the fixed-point weights q (not their CDF:
    the deterministic part needs the individual q_i).  step: how the R
    residual outputs are drawn on the residual weights -- "multinomial"
    (R sorted iid uniforms), "systematic" (one uniform, targets (k + u) / R)
    or "stratified" (targets (k + u_k) / R), the residual variants listed by
    Douc et al. (2005)."""
    n = len(q)
    d, R, r, _ = residual_parts(q)
    counts = np.array(d, dtype=np.int64)
    if R > 0:
        RQ = cdf(r)
        if step == "multinomial":
            P, D = multinomial_targets(R, philox.resample_u24(seed, t, R, stream))
            # multinomial_targets scales by its own count R: P = R (2 j + 1), D = R 2^25
        elif step == "systematic":
            P, D = systematic_targets(R, philox.systematic_u24(seed, t, stream))
        elif step == "stratified":
            P, D = stratified_targets(R, philox.resample_u24(seed, t, R, stream))
        else:
            raise ValueError(step)
        extra = select(RQ, P, D)
        counts += np.bincount(extra, minlength=n)
    return expand(counts)


def expand(counts):
    """Sorted ancestor array in which i appears counts[i] times."""
    return np.repeat(np.arange(len(counts), dtype=np.int64), np.asarray(counts, dtype=np.int64))


def offspring(a, n):
    """Replication counts R_i of the paper (Sec. 2.1) from ancestors."""
    return np.bincount(np.asarray(a, dtype=np.int64), minlength=n)


RESIDUAL_STEPS = {"residual": "multinomial", "residual_systematic": "systematic",
                  "residual_stratified": "stratified"}


def resample(scheme, lw, seed, t, stream=0):
    """Ancestors for the named scheme from raw log-weights."""
    q = quantise(lw)
    if scheme in RESIDUAL_STEPS:
        return residual(q, seed, t, stream, RESIDUAL_STEPS[scheme])
    Q = cdf(q)
    return {"systematic": systematic, "stratified": stratified,
            "multinomial": multinomial}[scheme](Q, seed, t, stream)


# ---- the plain real-weight definition (Sec. 2.1), no quantisation --------
#
# The schemes above run on exact fixed-point weights.  What they stand for
# is the textbook definition on the real normalised weights: the CDF
# C_i = w_0 + ... + w_i of w_i = exp(lw_i - m) in float64, the target of
# output k scaled to C_N (systematic C_N (k + u) / N, stratified
# C_N (k + u_k) / N, multinomial C_N u_(k)), and the ancestor
# a_k = min{i : C_i > U_k}.  The residual step (Douc et al. 2005) keeps
# floor(N W_i) copies of particle i and draws the other R = N - sum floor(N W_i)
# multinomially on the residual weights N W_i - floor(N W_i).  The uniforms
# are the same Philox midpoints (2j + 1) / 2^25 as above.  These functions are
# the pin of the fixed-point schemes: both must give the same ancestors except
# where a target lies within the quantisation error of a CDF boundary.

def plain_weights(lw):
    """w_i = exp(lw_i - max lw) in float64 (the largest weight is 1)."""
    lw = np.asarray(lw, dtype=np.float64)
    m = float(np.max(lw))
    if not math.isfinite(m):
        raise FloatingPointError("all log-weights are -inf or NaN")
    return np.exp(lw - m)


def plain_select(C, U):
    """a_k = min{i : C_i > U_k} on a float64 CDF C (non-decreasing).  A target
    at or above C_N (a rounding artefact) goes to the last particle with a
    positive weight, so that a zero weight is never selected."""
    C = np.asarray(C, dtype=np.float64)
    a = np.searchsorted(C, np.asarray(U, dtype=np.float64), side="right").astype(np.int64)
    last = int(np.flatnonzero(np.diff(np.concatenate([[0.0], C])) > 0)[-1])
    return np.minimum(a, last)


def _mid(j):
    return (2.0 * np.asarray(j, dtype=np.float64) + 1.0) / float(1 << 25)


def plain_resample(scheme, lw, seed, t, stream=0):
    """Ancestors of the named scheme on the float64 CDF of the real weights
    (sorted, like the fixed-point schemes)."""
    w = plain_weights(lw)
    n = w.shape[0]
    k = np.arange(n, dtype=np.float64)
    if scheme in RESIDUAL_STEPS:
        return _plain_residual(w, seed, t, stream, RESIDUAL_STEPS[scheme])
    C = np.cumsum(w)
    CN = C[-1]
    if scheme == "systematic":
        U = CN * (k + _mid(philox.systematic_u24(seed, t, stream))) / n
    elif scheme == "stratified":
        U = CN * (k + _mid(philox.resample_u24(seed, t, n, stream))) / n
    elif scheme == "multinomial":
        U = CN * np.sort(_mid(philox.resample_u24(seed, t, n, stream)))
    else:
        raise ValueError(scheme)
    return plain_select(C, U)


def plain_residual_parts(w):
    """floor(N W_i), R and the residual weights N W_i - floor(N W_i), float64."""
    n = w.shape[0]
    nw = n * (w / np.sum(w))
    d = np.floor(nw)
    return d.astype(np.int64), int(n - d.sum()), nw - d


def plain_residual_targets(R, seed, t, stream, step):
    """Targets of the R residual outputs as fractions of the residual total."""
    k = np.arange(R, dtype=np.float64)
    if step == "multinomial":
        return np.sort(_mid(philox.resample_u24(seed, t, R, stream)))
    if step == "systematic":
        return (k + _mid(philox.systematic_u24(seed, t, stream))) / R
    if step == "stratified":
        return (k + _mid(philox.resample_u24(seed, t, R, stream))) / R
    raise ValueError(step)


def _plain_residual(w, seed, t, stream, step="multinomial"):
    n = w.shape[0]
    d, R, r = plain_residual_parts(w)
    counts = d.copy()
    if R > 0:
        RC = np.cumsum(r)
        U = RC[-1] * plain_residual_targets(R, seed, t, stream, step)
        counts += np.bincount(plain_select(RC, U), minlength=n)
    return expand(counts)


# ---- the in-place ("j stays j") ancestor permutation (Sec. 4.1.2) -------
#
# The sampler's copy(N, copy_from) lets a resampling step say, for every new
# particle k, which old particle it copies.  Any arrangement of the ancestor
# multiset is the same resampled system; the in-place arrangement keeps
# every surviving particle in its own slot (copy_from[j] = j whenever
# particle j has offspring), so an in-place copy touches only the slots of
# particles without offspring.  Reading (the paper does not fix the order of
# the other slots): the extra copies, in increasing order of parent, fill the
# empty slots in increasing order.

def stay_permutation(ancestors):
    """copy_from with survivors in place, from any ancestor array."""
    a = np.sort(np.asarray(ancestors, dtype=np.int64))
    n = a.shape[0]
    o = np.bincount(a, minlength=n)
    out = np.arange(n, dtype=np.int64)
    empty = np.flatnonzero(o == 0)
    extras = np.repeat(np.arange(n, dtype=np.int64), np.maximum(o - 1, 0))
    assert empty.shape == extras.shape
    out[empty] = extras
    return out
