"""Negative log-likelihood, its gradient and the expected Fisher information (oracle).

Plain dense definitions, applied to the densified HODLR matrices K~ and K~_j.  The
hierarchical factorization (eq. one way factor, App. C) and the trace operations of
App. B reach these values exactly up to rounding (Sec. 4.2: "Both operations can be
conducted exactly"), so the oracle is the definition itself:
  NLL(theta)  = n/2 log(2 pi) + 1/2 log|K~| + 1/2 y^T K~^{-1} y          (eq. log-like approximated, negated)
  g_j         = dNLL/dtheta_j = 1/2 tr(K~^{-1} K~_j) - 1/2 y^T K~^{-1} K~_j K~^{-1} y
                                                                          (eq. score approximated, negated)
  I_ij        = 1/2 tr(K~^{-1} K~_i K~^{-1} K~_j)                         (eq. fisher info approximated)
Sign convention: the library returns the NLL and its gradient g = -S.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def nll(K, y):
    """Negative Gaussian log-likelihood with zero mean (eq. log-like)."""
    c, low = scipy.linalg.cho_factor(K, lower=True)
    logdet = 2.0 * np.sum(np.log(np.diag(c)))
    alpha = scipy.linalg.cho_solve((c, low), y)
    n = K.shape[0]
    return 0.5 * n * math.log(2.0 * math.pi) + 0.5 * logdet + 0.5 * float(y @ alpha)


def logdet(K):
    c, _ = scipy.linalg.cho_factor(K, lower=True)
    return 2.0 * float(np.sum(np.log(np.diag(c))))


def solve(K, y):
    return scipy.linalg.cho_solve(scipy.linalg.cho_factor(K, lower=True), y)


def grad(K, Ks, y):
    """dNLL/dtheta_j for the list of derivative matrices Ks (eq. score, negated)."""
    cf = scipy.linalg.cho_factor(K, lower=True)
    alpha = scipy.linalg.cho_solve(cf, y)
    g = []
    for Kj in Ks:
        tr = np.trace(scipy.linalg.cho_solve(cf, Kj))
        g.append(0.5 * tr - 0.5 * float(alpha @ (Kj @ alpha)))
    return np.array(g)


def trace_prod(A, B):
    """tr(A B) = sum_ij A_ij B_ji (the definition of the trace of a product, without forming
    A B)."""
    return float(np.sum(A * B.T))


def fisher(K, Ks):
    """Expected Fisher information I_ij = 1/2 tr(K^{-1} K_i K^{-1} K_j) (eq. fisher info)."""
    cf = scipy.linalg.cho_factor(K, lower=True)
    W = [scipy.linalg.cho_solve(cf, Kj) for Kj in Ks]
    p = len(Ks)
    F = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            F[i, j] = 0.5 * trace_prod(W[i], W[j])
    return F


def traces(K, Ms):
    """tr(K^{-1} M_i) and tr(K^{-1} M_i K^{-1} M_j) for the list Ms (App. B.3 values)."""
    cf = scipy.linalg.cho_factor(K, lower=True)
    W = [scipy.linalg.cho_solve(cf, M) for M in Ms]
    t = np.array([np.trace(Wi) for Wi in W])
    f = np.array([[trace_prod(Wi, Wj) for Wj in W] for Wi in W])
    return t, f


def evaluate(H, y_tree, params=("sigma2", "ell", "kappa", "tau2")):
    """NLL, gradient and Fisher of the HODLR approximation H (tree-ordered y).

    The same definitions as nll(), grad() and fisher(), with one Cholesky factorization and
    one solve K~^{-1} K~_j per parameter shared by the gradient and the Fisher matrix."""
    K = H.densify("K")
    cf = scipy.linalg.cho_factor(K, lower=True)
    n = K.shape[0]
    logdet_k = 2.0 * float(np.sum(np.log(np.diag(cf[0]))))
    alpha = scipy.linalg.cho_solve(cf, y_tree)
    f = 0.5 * n * math.log(2.0 * math.pi) + 0.5 * logdet_k + 0.5 * float(y_tree @ alpha)
    del K
    W, g = [], []
    for p in params:
        Kj = H.densify(p)
        Wj = scipy.linalg.cho_solve(cf, Kj)
        g.append(0.5 * np.trace(Wj) - 0.5 * float(alpha @ (Kj @ alpha)))
        W.append(Wj)
        del Kj
    F = np.zeros((len(params), len(params)))
    for i in range(len(params)):
        for j in range(len(params)):
            F[i, j] = 0.5 * trace_prod(W[i], W[j])
    return f, np.array(g), F
