"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline may import this module. The CUDA path carries its own generator,
written separately from the same published definition.

Philox4x32-10 is defined in Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter and a 2 x 32-bit
key; each of the 10 rounds multiplies counter words 0 and 2 by fixed 32-bit
constants, keeps both halves of the 64-bit products, and mixes them with the
other two counter words and the key; the key is bumped by two Weyl constants
between rounds.

The auxiliary fields of Eq. 2 (Sec. II) are unit normals x_g. Each walker
draws them from the counter (g // 4, walker, step, 4 * run_id + stream) with
stream 0; stream 1 supplies the comb offset of population control. The key is
the 64-bit seed split into (low word, high word). The four words give two
Box-Muller pairs, x[4q], x[4q+1] from words 0, 1 and x[4q+2], x[4q+3] from
words 2, 3, with u = (r + 1/2) / 2**32 so that u is never 0.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

STREAM_FIELDS = 0
STREAM_COMB = 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds; array inputs broadcast. Returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK
                      for c in np.broadcast_arrays(c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def uniform_open01(r):
    """Map a uint32 word to (0, 1): (r + 1/2) * 2**-32, exact in float64."""
    return (np.asarray(r, dtype=np.float64) + 0.5) * (2.0 ** -32)


def box_muller(ra, rb):
    """Two independent unit normals from two uint32 words."""
    ua = uniform_open01(ra)
    ub = uniform_open01(rb)
    rad = np.sqrt(-2.0 * np.log(ua))
    return rad * np.cos(2.0 * np.pi * ub), rad * np.sin(2.0 * np.pi * ub)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def gaussian_fields(seed, run_id, step, walkers, n_chol):
    """Auxiliary fields x[w, g] ~ N(0, 1) for the given walker indices at a step."""
    walkers = np.asarray(walkers, dtype=np.int64)
    nq = (n_chol + 3) // 4
    q = np.arange(nq, dtype=np.uint64)[None, :]
    w = walkers.astype(np.uint64)[:, None]
    k0, k1 = _key(seed)
    r = philox4x32_10(q, w, np.uint64(step),
                      np.uint64(4 * run_id + STREAM_FIELDS), k0, k1)
    z0, z1 = box_muller(r[0], r[1])
    z2, z3 = box_muller(r[2], r[3])
    x = np.stack([z0, z1, z2, z3], axis=-1).reshape(walkers.size, 4 * nq)
    return x[:, :n_chol]


def comb_uniform(seed, run_id, step):
    """Comb offset u in (0, 1) for population control at a step (stream 1)."""
    k0, k1 = _key(seed)
    r = philox4x32_10(0, 0, np.uint64(step),
                      np.uint64(4 * run_id + STREAM_COMB), k0, k1)
    return float(uniform_open01(r[0]))
