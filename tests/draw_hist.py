"""Histogram of the 24-bit resampling draws j_k of a whole step, from the
oracle's Philox (oracle.philox.resample_u24's draws, computed a range of
Philox calls at a time so that N = 2^30 fits in host memory).  A worker
function for a spawned process pool: numpy and the oracle only."""
import numpy as np

from oracle import philox as ophilox

CHUNK = 1 << 20  # Philox calls (4 draws each) per numpy pass


def hist_range(args):
    """Counts of each 24-bit value among the draws of Philox calls
    [c0, c1) at (seed, t): call c gives j_{4c}, ..., j_{4c+3}."""
    seed, t, c0, c1 = args
    h = np.zeros(1 << 24, dtype=np.int64)
    for a in range(c0, c1, CHUNK):
        b = min(a + CHUNK, c1)
        w = ophilox.draw_words(seed, np.arange(a, b, dtype=np.int64), t, ophilox.TAG_RESAMPLE, 0, 0)
        h += np.bincount(ophilox.u24(w).reshape(-1), minlength=1 << 24)
    return h


def draw_counts(seed, t, n, pool, parts):
    """Counts of each 24-bit value among j_0 .. j_{n-1} (n a multiple of 4)."""
    assert n % 4 == 0
    calls = n // 4
    bounds = [calls * p // parts for p in range(parts + 1)]
    h = np.zeros(1 << 24, dtype=np.int64)
    for part in pool.imap_unordered(hist_range, [(seed, t, bounds[p], bounds[p + 1]) for p in range(parts)]):
        h += part
    return h
