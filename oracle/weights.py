"""Weights, normaliser, ESS, normalising-constant ratio and the resample test.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed (float64 throughout):
* normalised weights W_i proportional to w_i with sum 1 (Sec. 2.1, the
  estimator phi-hat-3);
* ESS = 1 / sum_i W_i^2 (Sec. 2.1, ESS definition);
* the ratio of normalising constants Z_t / Z_{t-1} is estimated by
  sum_i W_{t-1,i} w_t,i (Sec. 2.2), i.e. in logs by the log-sum-exp of
  log W_{t-1,i} + log w_t,i;
* resampling is done when ESS / N is below the threshold; threshold >= 1
  always resamples, threshold <= 0 never does (Sec. 4.1.3, Sampler
  constructor).  Reading: "below" is a strict "<".

Representation (a reading, the same on both sides): the stored raw
log-weight at iteration t is lw_t,i = log W_{t-1,i} + log w_t,i, so its
log-sum-exp L_t is at once the log-normaliser of W_t and the log of the
estimated ratio Z_t / Z_{t-1}; log W_{t-1,i} is lw_{t-1,i} - L_{t-1}, or
-log N after a resampling step (equal weights 1/N).

Parity pins: sum W = 1, ESS = N for equal weights, 1 <= ESS <= N, agreement
with the naive un-shifted sum on well-scaled inputs (tests/test_oracle_weights.py).
"""
import math

import numpy as np


def log_sum_exp(lw):
    """m + log sum exp(lw - m), m = max lw.  Returns (m, L)."""
    lw = np.asarray(lw, dtype=np.float64)
    m = float(np.max(lw))
    if not math.isfinite(m):
        raise FloatingPointError("all log-weights are -inf or NaN")
    return m, m + math.log(float(np.sum(np.exp(lw - m))))


def normalised(lw):
    """Normalised weights W_i = exp(lw_i - L)."""
    _, L = log_sum_exp(lw)
    return np.exp(np.asarray(lw, dtype=np.float64) - L)


def ess(lw):
    """Effective sample size 1 / sum W_i^2."""
    W = normalised(lw)
    return 1.0 / float(np.sum(W * W))


def weighted_mean(lw, h):
    """Importance-sampling estimate sum_i W_i h(X_i) (phi-hat-3)."""
    return float(np.sum(normalised(lw) * np.asarray(h, dtype=np.float64)))


def resample_decision(ess_value, n, threshold):
    """True when resampling is due (strict ESS < threshold * N)."""
    if threshold >= 1.0:
        return True
    if threshold <= 0.0:
        return False
    return ess_value < threshold * n


def previous_log_weight(lw_prev, L_prev, resampled_prev, n):
    """log W_{t-1,i}: normalised previous log-weights, or -log N after a
    resampling step."""
    if resampled_prev:
        return np.full(n, -math.log(n))
    return np.asarray(lw_prev, dtype=np.float64) - L_prev
