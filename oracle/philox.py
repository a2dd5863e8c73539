"""Gaussian sampling matrices for the level sketches (oracle).

Alg. 1 step 1 draws a Gaussian sampling matrix; Sec. 3.2.2 makes it *patterned*
(non-zero only on the rows of the right child of every block pair at the level) and
Sec. 3.3 requires it to stay fixed across theta.  A counter-based generator makes
the draw a pure function of (seed, level, column, row), so the CPU oracle and the
GPU draw identical integers.

Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written here from its published definition:
  round:  (c0,c1,c2,c3) <- (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
  key schedule between rounds: k0 += W0, k1 += W1 (mod 2^32); 10 rounds.
Counter words: c0 = row position i, c1 = column j, c2 = level l, c3 = stream id.
Key: (seed mod 2^32, seed >> 32).
Normal deviate (reading): u1 = ((w0>>5)*2^26 + (w1>>6) + 1) * 2^-53 in (0, 1],
u2 = ((w2>>5)*2^26 + (w3>>6)) * 2^-53 in [0, 1), z = sqrt(-2 ln u1) cos(2 pi u2).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; arguments are integer arrays/scalars < 2^32."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    for r in range(10):
        if r:
            k0 = np.uint64((int(k0) + W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + W1) & 0xFFFFFFFF)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def normal(rows, col, level, stream, seed):
    """Standard normal deviates for counters (rows, col, level, stream)."""
    w0, w1, w2, w3 = philox4x32_10(rows, col, level, stream, seed & 0xFFFFFFFF, seed >> 32)
    two26 = np.float64(67108864.0)
    u1 = ((w0 >> np.uint64(5)).astype(np.float64) * two26
          + (w1 >> np.uint64(6)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = ((w2 >> np.uint64(5)).astype(np.float64) * two26
          + (w3 >> np.uint64(6)).astype(np.float64)) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def level_probe(tree, level: int, ncols: int, seed: int, stream: int = 0) -> np.ndarray:
    """Patterned probe R^(l) (N x ncols): Gaussian on right-child rows, zero elsewhere.

    Sec. 3.2.2 ("Processing level 1/2"): rows of the left child I_1 are zero and rows
    of the right child carry i.i.d. standard normal entries, for every block pair.
    """
    R = np.zeros((tree.N, ncols))
    rows = []
    for (_, _), (lo2, hi2) in tree.pairs(level):
        rows.append(np.arange(lo2, hi2))
    rows = np.concatenate(rows).astype(np.uint64)
    for j in range(ncols):
        R[rows.astype(np.int64), j] = normal(rows, j, level, stream, seed)
    return R
