"""Ordering and cluster tree (oracle).

Follows Sec. 5.2 (observations ordered by a KD-tree binary spatial partition so that
off-diagonal blocks couple well-separated groups) and the index sets I_i^(l) of
Sec. 3.2.2 (contiguous halves of the parent range at every level).

Readings:
  * 1-D: natural order of the interior nodes x_i = i/(G+1).
  * 2-D: Morton (Z) order with x-index bit b at key bit 2b and y-index bit b at key
    bit 2b+1, ascending; on a 2^q x 2^q grid this is the KD tree with median splits
    alternating y then x.
  * A node covering positions [lo, hi) splits at mid = lo + (hi - lo) // 2.  tau is the
    smallest integer with ceil(Ns / 2^tau) <= spatial leaf size; every node is split
    exactly tau times, so all leaves are at depth tau.
  * Bivariate (nvar = 2): the tree is built over the Ns spatial points; within each
    spatial leaf the matrix rows are [variable 1 of its points, variable 2 of the same
    points].  Natural layout of a bivariate vector is [y1 (Ns); y2 (Ns)].
"""
from __future__ import annotations

import math

import numpy as np


def spatial_order(dim: int, G: int) -> np.ndarray:
    """Natural grid index of the point at each spatial tree position."""
    if dim == 1:
        return np.arange(G, dtype=np.int64)
    iy, ix = np.divmod(np.arange(G * G, dtype=np.int64), G)   # natural p = iy*G + ix
    key = np.zeros(G * G, dtype=np.int64)
    nbits = max(1, math.ceil(math.log2(G)))
    for b in range(nbits):
        key |= ((ix >> b) & 1) << (2 * b)
        key |= ((iy >> b) & 1) << (2 * b + 1)
    return np.argsort(key, kind="stable").astype(np.int64)


def n_levels(n_points: int, leaf_points: int) -> int:
    """Smallest tau with ceil(n_points / 2^tau) <= leaf_points."""
    tau = 0
    while -(-n_points // (1 << tau)) > leaf_points:
        tau += 1
    return tau


class Tree:
    """Cluster tree over matrix positions 0..N-1 (N = nvar * Ns)."""

    def __init__(self, dim: int, G: int, nvar: int, leaf_rows: int):
        if leaf_rows % nvar:
            raise ValueError("leaf size must be a multiple of the number of variables")
        self.dim, self.G, self.nvar = dim, G, nvar
        self.Ns = G ** dim
        self.N = nvar * self.Ns
        self.tau = n_levels(self.Ns, leaf_rows // nvar)
        # spatial bounds per depth: list of (lo, hi)
        bounds = [[(0, self.Ns)]]
        for _ in range(self.tau):
            nxt = []
            for lo, hi in bounds[-1]:
                mid = lo + (hi - lo) // 2
                nxt.append((lo, mid))
                nxt.append((mid, hi))
            bounds.append(nxt)
        self.spatial_bounds = bounds
        # matrix-row bounds per depth
        self.bounds = [[(nvar * lo, nvar * hi) for lo, hi in lvl] for lvl in bounds]
        sp = spatial_order(dim, G)
        if nvar == 1:
            perm = sp
        else:
            parts = []
            for lo, hi in bounds[-1]:
                parts.append(sp[lo:hi])
                parts.append(self.Ns + sp[lo:hi])
            perm = np.concatenate(parts)
        self.perm = perm.astype(np.int64)          # perm[position] = natural index

    def pairs(self, level: int):
        """Block pairs (c1, c2) of HODLR level `level` (1 = coarsest), as row ranges."""
        out = []
        kids = self.bounds[level]
        for b in range(0, len(kids), 2):
            out.append((kids[b], kids[b + 1]))
        return out

    def leaves(self):
        return self.bounds[self.tau]

    def to_tree(self, x_nat: np.ndarray) -> np.ndarray:
        return x_nat[self.perm]

    def to_natural(self, x_tree: np.ndarray) -> np.ndarray:
        out = np.empty_like(x_tree)
        out[self.perm] = x_tree
        return out
