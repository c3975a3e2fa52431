"""Philox4x32-10 and the variate transforms used by every SMC step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper gives every particle its own independent counter-based random
stream (Sec. 3.4, Third-party dependencies; Sec. 4.1.7, RngSet).  The method
draws its random numbers from Philox4x32-10 as published by Salmon, Moraes,
Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11):

* state: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1);
* one round maps (c0, c1, c2, c3) to
  (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
  with M0 = 0xD2511F53 and M1 = 0xCD9E8D57 (32x32 -> 64-bit products);
* between rounds the key is bumped by the Weyl constants
  (0x9E3779B9, 0xBB67AE85);
* ten rounds.

Counter assignment (a convention of this implementation, documented beside
the C ABI as well):  key = (low 32 bits of seed, high 32 bits of seed);
counter = (index, iteration t, purpose tag | stream << 16, draw).

Transforms
* uniform: j = x >> 8 (24 bits), u = (j + 1) / 2^24, in (0, 1] and exactly
  representable in both float32 and float64 (the paper's Metropolis step
  takes a (0, 1] uniform, Sec. 5.2.4); resampling uses j through the exact
  rational (2j + 1) / 2^25 in (0, 1) instead (``oracle.resample``);
* normal pairs: Box-Muller, z0 = sqrt(-2 ln u0) cos(2 pi u1),
  z1 = sqrt(-2 ln u0) sin(2 pi u1) (the paper leaves the normal generator to
  the standard library, whose algorithm is implementation-defined);
* exponential: -ln u.

Parity pins: published Philox4x32-10 known-answer vectors
(tests/golden/philox4x32_10_kat.txt); moments / Kolmogorov-Smirnov tests of
the transforms.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

# purpose tags (counter word c2, low 16 bits)
TAG_INIT = 1
TAG_MOVE = 2
TAG_RESAMPLE = 3
TAG_MH_MU = 4
TAG_MH_LAMBDA = 5
TAG_MH_WEIGHT = 6
TAG_MALA = 7
TAG_RESIDUAL = 8

# draw index of the Metropolis-Hastings acceptance uniform (word 0)
DRAW_MH_UNIFORM = 16


def philox4x32_10(ctr, key):
    """Ten Philox4x32 rounds.

    ctr: (n, 4) integer array (values < 2^32); key: (2,) or (n, 2).
    Returns an (n, 4) uint32 array.
    """
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint64)
    if k.ndim == 1:
        k = np.broadcast_to(k, (c.shape[0], 2))
    c0, c1, c2, c3 = (c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy())
    k0, k1 = k[:, 0].copy(), k[:, 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0            # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def key_of(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def counters(index, t, tag, stream=0, draw=0):
    """Counter array for a vector of indices (the other words broadcast)."""
    index = np.asarray(index, dtype=np.uint64).reshape(-1)
    n = index.shape[0]
    c = np.empty((n, 4), dtype=np.uint64)
    c[:, 0] = index
    c[:, 1] = np.uint64(t)
    c[:, 2] = np.uint64((int(tag) & 0xFFFF) | ((int(stream) & 0xFFFF) << 16))
    c[:, 3] = np.asarray(draw, dtype=np.uint64)
    return c


def draw_words(seed, index, t, tag, stream=0, draw=0):
    """(n, 4) uint32 Philox output for the given particle indices."""
    return philox4x32_10(counters(index, t, tag, stream, draw), key_of(seed))


def u24(x):
    """24-bit integer j = x >> 8 of a 32-bit word."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.int64)


def uniform(x):
    """u = (j + 1) / 2^24 with j = x >> 8; exact in float32 and float64."""
    return (u24(x).astype(np.float64) + 1.0) * 2.0 ** -24


def box_muller(u0, u1):
    r = np.sqrt(-2.0 * np.log(u0))
    return r * np.cos(2.0 * np.pi * u1), r * np.sin(2.0 * np.pi * u1)


def normals(seed, index, t, tag, count, stream=0):
    """`count` standard normals per index, shape (count, n).

    Normal m uses call draw = m // 4; the pair (w0, w1) feeds normals
    m % 4 in {0, 1} and (w2, w3) feeds m % 4 in {2, 3}.
    """
    index = np.asarray(index).reshape(-1)
    out = np.empty((count, index.shape[0]), dtype=np.float64)
    for call in range((count + 3) // 4):
        w = draw_words(seed, index, t, tag, stream, draw=call)
        za, zb = box_muller(uniform(w[:, 0]), uniform(w[:, 1]))
        zc, zd = box_muller(uniform(w[:, 2]), uniform(w[:, 3]))
        for m, z in enumerate((za, zb, zc, zd)):
            if 4 * call + m < count:
                out[4 * call + m] = z
    return out


def exponentials(seed, index, t, tag, count, first_draw, stream=0):
    """`count` Exp(1) variates per index, shape (count, n): -ln u, word m % 4
    of call draw = first_draw + m // 4."""
    index = np.asarray(index).reshape(-1)
    out = np.empty((count, index.shape[0]), dtype=np.float64)
    for m in range(count):
        w = draw_words(seed, index, t, tag, stream, draw=first_draw + m // 4)
        out[m] = -np.log(uniform(w[:, m % 4]))
    return out


def resample_u24(seed, t, count, stream=0):
    """The 24-bit integers j_k, k < count, that drive stratified,
    multinomial and residual resampling at iteration t: word k % 4 of the
    call with counter (k // 4, t, TAG_RESAMPLE | stream << 16, 0)."""
    k = np.arange(count, dtype=np.int64)
    w = draw_words(seed, k // 4, t, TAG_RESAMPLE, stream, 0)
    return u24(w[np.arange(count), k % 4])


def systematic_u24(seed, t, stream=0):
    """The single 24-bit integer j of systematic resampling at iteration t
    (word 0 of the call with counter (0, t, TAG_RESAMPLE | stream << 16, 0))."""
    w = draw_words(seed, [0], t, TAG_RESAMPLE, stream, 0)
    return int(u24(w[0, 0]))
