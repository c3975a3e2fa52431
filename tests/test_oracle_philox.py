"""Pins of the oracle's Philox4x32-10 and variate transforms."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(h, 16) for h in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_published_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10([ctr], key)[0]
        assert [int(x) for x in got] == out


def test_vectorised_matches_rowwise():
    ctr = np.array([[i, 7, 3, 1] for i in range(5)])
    key = [123, 456]
    many = philox.philox4x32_10(ctr, key)
    for i in range(5):
        assert np.array_equal(many[i], philox.philox4x32_10([ctr[i]], key)[0])


def test_uniform_exact_and_open_interval():
    x = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.uniform(x)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24
    assert u[2] == 2 * 2.0 ** -24
    assert u[3] == 1.0
    assert np.all(np.float32(u) == u)          # exactly representable in float32


def test_normals_distribution():
    z = philox.normals(42, np.arange(50000), 3, philox.TAG_MOVE, 4)
    flat = z.reshape(-1)
    assert abs(flat.mean()) < 5 / np.sqrt(flat.size)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    # the four lanes are uncorrelated
    c = np.corrcoef(z)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(z.shape[1])


def test_exponentials_distribution():
    e = philox.exponentials(7, np.arange(40000), 0, philox.TAG_INIT, 3, first_draw=4)
    flat = e.reshape(-1)
    assert stats.kstest(flat, "expon").pvalue > 1e-4


def test_streams_differ_by_every_counter_word():
    base = philox.draw_words(1, [5], 2, philox.TAG_MOVE, 0, 0)[0]
    for kw in (dict(index=[6]), dict(t=3), dict(tag=philox.TAG_INIT), dict(stream=1), dict(draw=1)):
        args = dict(index=[5], t=2, tag=philox.TAG_MOVE, stream=0, draw=0)
        args.update(kw)
        w = philox.draw_words(1, args["index"], args["t"], args["tag"], args["stream"], args["draw"])[0]
        assert not np.array_equal(w, base)
    assert not np.array_equal(philox.draw_words(2, [5], 2, philox.TAG_MOVE)[0], base)


def test_draw_histogram_helper_counts_the_resampling_draws():
    """tests/draw_hist.py (the large-N tests' draw histogram, computed a
    range of Philox calls at a time) counts exactly the draws of
    resample_u24, split over any number of parts."""
    import draw_hist

    class Serial:
        imap_unordered = staticmethod(map)

    n = 4 * 5003
    want = np.bincount(philox.resample_u24(3, 7, n), minlength=1 << 24)
    for parts in (1, 3, 8):
        assert np.array_equal(draw_hist.draw_counts(3, 7, n, Serial(), parts), want)
