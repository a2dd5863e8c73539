"""Matrix-free randomized HODLR construction and its derivative (oracle).

Follows, step by step and in the paper's order:
  * Alg. 1 (randomized low-rank approximation): Gaussian sampling, Y = B Omega, QR with
    column pivoting, Q, then B^T Q;
  * Sec. 3.2.2 (construction from matrix-vector products): per level l = 1..tau, the
    patterned probe R^(l) (eq. lvl1 sample1 / lvl2 sample1), peeling of all coarser
    levels' low-rank blocks, QR of the c1-rows of the sample, the second patterned
    probe S^(l) = [Q; 0] (eq. lvl1 sample2 / lvl2 sample2), B~ = (c2-rows of the result),
    B^ = Q B~^T (eq. lowrnkB11 / lowrnkB212); leaf level by stacked identities
    (eq. leaf sample);
  * Sec. 3.3 (differentiating the approximation) with the probes fixed: dY from the
    differentiated products (eq. db1r1, eq. lvl2 sample1 diff), Alg. 2 for dQ, dB~ from
    eq. prod-rule-2 / eq. lvl2 sample2 diff / eq. tmp2, dB^ = dQ B~^T + Q dB~^T
    (eq. diff low-rank, eq. lvl2 block1 diff), leaf derivatives from eq. diag diff.

Readings (the paper is silent on these):
  * Alg. 1's sampling matrix for B in R^{p x q} is q x k (printed p x k).
  * c probe columns per level; the kept rank r of a block is the number of leading
    |R_ii| of the pivoted QR above max(tol, guard) * |R_11|, capped at `cap`; the
    guard keeps Alg. 2's R invertible (Alg. 2 assumes full column rank).
  * Q is the Q factor of the (unpivoted) QR of Y[:, J], J = pivots[:r], with a positive
    diagonal of R, so Q is unique; R is that QR's triangular factor.  J is frozen when
    differentiating.
  * Extracted leaf blocks are symmetrised, A_b = (E_b + E_b^T)/2.
  * dK~/dsigma2 = (K~ - tau2 I)/sigma2 and dK~/dtau2 = I (the construction is linear in
    sigma2 with a scale-invariant rank rule, and tau2 I never reaches an off-diagonal
    row of a sketch); the general sweep may also be run for sigma2 to check this.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .philox import level_probe


class Level:
    """Low-rank factors of one HODLR level: per block pair (Q, B~), B^ = Q B~^T."""

    def __init__(self):
        self.Q, self.Bt, self.J, self.R, self.rank = [], [], [], [], []
        self.width = 0


class Hodlr:
    def __init__(self, tree, theta):
        self.tree = tree
        self.theta = tuple(float(t) for t in theta)
        self.levels = []          # index l-1
        self.leaves = []
        self.dlevels = {}         # param -> list of per-level (dQ list, dBt list)
        self.dleaves = {}
        self.napply = 0           # number of K or K_j vector products (columns)

    # ------------------------------------------------------------------ products
    def offdiag_apply(self, X, levels, deriv=None):
        """Sum over the given levels of (off-diagonal part) X, or its derivative."""
        out = np.zeros_like(X)
        for l in levels:
            L = self.levels[l - 1]
            for p, ((a1, b1), (a2, b2)) in enumerate(self.tree.pairs(l)):
                Q, Bt = L.Q[p], L.Bt[p]
                if Q.shape[1] == 0:
                    continue
                if deriv is None:
                    out[a1:b1] += Q @ (Bt.T @ X[a2:b2])
                    out[a2:b2] += Bt @ (Q.T @ X[a1:b1])
                else:
                    dQ, dBt = self.dlevels[deriv][l - 1][0][p], self.dlevels[deriv][l - 1][1][p]
                    out[a1:b1] += dQ @ (Bt.T @ X[a2:b2]) + Q @ (dBt.T @ X[a2:b2])
                    out[a2:b2] += Bt @ (dQ.T @ X[a1:b1]) + dBt @ (Q.T @ X[a1:b1])
        return out

    # ------------------------------------------------------------------ dense form
    def densify(self, which="K"):
        N = self.tree.N
        sigma2, _, _, tau2 = self.theta
        if which == "tau2" and which not in self.dleaves:
            return np.eye(N)
        if which == "sigma2" and which not in self.dleaves:
            return (self.densify("K") - tau2 * np.eye(N)) / sigma2
        D = np.zeros((N, N))
        leaves = self.leaves if which == "K" else self.dleaves[which]
        for (lo, hi), A in zip(self.tree.leaves(), leaves):
            D[lo:hi, lo:hi] = A
        for l in range(1, self.tree.tau + 1):
            L = self.levels[l - 1]
            for p, ((a1, b1), (a2, b2)) in enumerate(self.tree.pairs(l)):
                if which == "K":
                    blk = L.Q[p] @ L.Bt[p].T
                else:
                    dQ = self.dlevels[which][l - 1][0][p]
                    dBt = self.dlevels[which][l - 1][1][p]
                    blk = dQ @ L.Bt[p].T + L.Q[p] @ dBt.T
                D[a1:b1, a2:b2] = blk
                D[a2:b2, a1:b1] = blk.T
        return D

    def ranks(self):
        return [list(L.rank) for L in self.levels]

    def pivots(self):
        return [list(L.J) for L in self.levels]


def _qr_positive(Y):
    """Unpivoted economic QR with positive diagonal of R (unique Q)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def build(model, tree, theta, *, c, cap, tol=0.0, guard=1e-7, seed=1, stream=0,
          params=("ell", "kappa"), frozen=None):
    """Construct K~(theta) and the derivative HODLR matrices K~_j for j in `params`.

    model: oracle.physics.Model; tree: oracle.tree.Tree; frozen: optional per-level
    list of per-pair pivot sets J (then no pivoted QR is taken).
    """
    H = Hodlr(tree, theta)
    perm = tree.perm
    N = tree.N

    def Kapp(X, which):
        H.napply += X.shape[1]
        Xn = np.zeros_like(X)
        Xn[perm] = X
        return model.apply(Xn, theta, which)[perm]

    for j in params:
        H.dlevels[j] = []

    for l in range(1, tree.tau + 1):
        pairs = tree.pairs(l)
        coarser = range(1, l)
        Lv = Level()
        # --- sample the column spaces of the level's blocks: (K - sum_{l'<l} H^(l')) R^(l)
        R = level_probe(tree, l, c, seed, stream)
        KR = {"K": Kapp(R, "K")}
        Y = KR["K"] - H.offdiag_apply(R, coarser)
        for p, ((a1, b1), (a2, b2)) in enumerate(pairs):
            Yb = Y[a1:b1]
            if frozen is not None:
                J = np.asarray(frozen[l - 1][p], dtype=np.int64)
            else:
                _, Rp, piv = scipy.linalg.qr(Yb, mode="economic", pivoting=True)
                d = np.abs(np.diag(Rp))
                r = 0
                if d.size and d[0] > 0.0:
                    thr = max(tol, guard) * d[0]
                    while r < d.size and d[r] > thr:
                        r += 1
                r = min(r, cap)
                J = np.asarray(piv[:r], dtype=np.int64)
            Q, Rj = _qr_positive(Yb[:, J]) if J.size else (np.zeros((b1 - a1, 0)), np.zeros((0, 0)))
            Lv.Q.append(Q)
            Lv.R.append(Rj)
            Lv.J.append(J)
            Lv.rank.append(int(J.size))
        w = max(Lv.rank) if Lv.rank else 0
        Lv.width = w
        # --- project: (K - sum H) S^(l), S^(l) = [Q; 0] per pair, B~ = c2-rows
        S = np.zeros((N, w))
        for p, ((a1, b1), _) in enumerate(pairs):
            S[a1:b1, :Lv.rank[p]] = Lv.Q[p]
        Z = Kapp(S, "K") - H.offdiag_apply(S, coarser)
        for p, (_, (a2, b2)) in enumerate(pairs):
            Lv.Bt.append(Z[a2:b2, :Lv.rank[p]].copy())
        H.levels.append(Lv)
        # --- differentiate the level (Sec. 3.3) for every requested parameter
        for j in params:
            dY_all = Kapp(R, j) - H.offdiag_apply(R, coarser, deriv=j)
            dQs, dBts = [], []
            for p, ((a1, b1), _) in enumerate(pairs):
                Q, Rj, J = Lv.Q[p], Lv.R[p], Lv.J[p]
                if J.size == 0:
                    dQs.append(np.zeros_like(Q))
                    continue
                dY = dY_all[a1:b1][:, J]
                # Alg. 2 step 1: Y' = Q^T dY R^{-1}
                dYRi = scipy.linalg.solve_triangular(Rj, dY.T, trans="T", lower=False).T
                Yp = Q.T @ dYRi
                # step 2: Y' = dOmega + dR R^{-1}, dOmega skew, dR R^{-1} upper triangular
                Lo = np.tril(Yp, -1)
                dOmega = Lo - Lo.T
                # step 3: dQ = Q dOmega + (I - Q Q^T) dY R^{-1}
                dQs.append(Q @ dOmega + (dYRi - Q @ (Q.T @ dYRi)))
            H.dlevels[j].append((dQs, dBts))
            dS = np.zeros((N, w))
            for p, ((a1, b1), _) in enumerate(pairs):
                dS[a1:b1, :Lv.rank[p]] = dQs[p]
            dZ = (Kapp(S, j) - H.offdiag_apply(S, coarser, deriv=j)
                  + Kapp(dS, "K") - H.offdiag_apply(dS, coarser))
            for p, (_, (a2, b2)) in enumerate(pairs):
                dBts.append(dZ[a2:b2, :Lv.rank[p]].copy())

    # --- leaf level: (K - sum_all H) [I; I; ...; I]
    leaves = tree.leaves()
    nl = max(hi - lo for lo, hi in leaves)
    S_leaf = np.zeros((N, nl))
    for lo, hi in leaves:
        S_leaf[lo:hi, :hi - lo] = np.eye(hi - lo)
    all_levels = range(1, tree.tau + 1)
    E = Kapp(S_leaf, "K") - H.offdiag_apply(S_leaf, all_levels)
    for lo, hi in leaves:
        Ab = E[lo:hi, :hi - lo]
        H.leaves.append(0.5 * (Ab + Ab.T))
    for j in params:
        dE = Kapp(S_leaf, j) - H.offdiag_apply(S_leaf, all_levels, deriv=j)
        H.dleaves[j] = []
        for lo, hi in leaves:
            Ab = dE[lo:hi, :hi - lo]
            H.dleaves[j].append(0.5 * (Ab + Ab.T))
    return H


def napply_formula(H, c, nderiv=2):
    """Number of K / K_j vector products of one build (the O(k tau) count of Sec. 3.2.2
    and Sec. 3.3).  Per level: K R^(l) and K S^(l) (c + w columns), and per derivative
    K_j R^(l), K_j S^(l), K dS^(l) (c + 2w columns), w = the level's widest kept rank;
    leaf level: (1 + nderiv) * leaf size."""
    n = 0
    for L in H.levels:
        n += (1 + nderiv) * c + (1 + 2 * nderiv) * L.width
    nl = max(hi - lo for lo, hi in H.tree.leaves())
    return n + (1 + nderiv) * nl
