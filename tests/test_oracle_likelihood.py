"""Pins of the oracle's NLL, gradient, Fisher information (eq. log-like / score / fisher info)
and Fisher scoring."""
import math

import numpy as np
import scipy.optimize

from oracle import hodlr, likelihood, scoring
from oracle.physics import Model
from oracle.tree import Tree

THETA = (1.0, 0.1, 5.0, 1e-3)
PARAMS = ("sigma2", "ell", "kappa", "tau2")


def test_nll_closed_form_identity_covariance():
    y = np.arange(5.0)
    val = likelihood.nll(2.0 * np.eye(5), y)
    assert math.isclose(val, 2.5 * math.log(2 * math.pi) + 2.5 * math.log(2.0) + 0.25 * float(y @ y),
                        rel_tol=1e-14)


def test_gradient_matches_finite_differences_of_nll():
    m = Model(1, 40, 1, 1.5)
    y = np.random.default_rng(1).standard_normal(40)
    g = likelihood.grad(m.dense_K(THETA), [m.dense_K(THETA, p) for p in PARAMS], y)
    for j in range(4):
        h = 1e-6 * THETA[j]
        tp = list(THETA); tm = list(THETA)
        tp[j] += h; tm[j] -= h
        fd = (likelihood.nll(m.dense_K(tp), y) - likelihood.nll(m.dense_K(tm), y)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(abs(g[j]), 1e-8 * np.abs(g).max()), j


def test_fisher_closed_form_scale_family():
    # K(s) = s K0: I_ss = n / (2 s^2)
    K0 = Model(1, 30, 1, 0.5).dense_K(THETA)
    s = 2.5
    F = likelihood.fisher(s * K0, [K0])
    assert math.isclose(F[0, 0], 30 / (2 * s * s), rel_tol=1e-12)


def test_fisher_is_covariance_of_score():
    # expected Fisher information = E[g g^T] for y ~ N(0, K) (Monte Carlo, 40000 draws)
    m = Model(1, 12, 1, 1.5)
    th = (1.0, 0.2, 3.0, 0.05)
    K = m.dense_K(th)
    Ks = [m.dense_K(th, p) for p in PARAMS]
    F = likelihood.fisher(K, Ks)
    rng = np.random.default_rng(3)
    Lc = np.linalg.cholesky(K)
    Y = Lc @ rng.standard_normal((12, 40000))
    Ki = np.linalg.inv(K)
    A = Ki @ Y
    G = np.stack([0.5 * np.trace(Ki @ Kj) - 0.5 * np.einsum("in,ij,jn->n", A, Kj, A) for Kj in Ks])
    emp = G @ G.T / Y.shape[1]
    d = np.sqrt(np.diag(F))
    assert np.abs((emp - F) / np.outer(d, d)).max() < 0.05


def test_leaf_only_tree_equals_dense():
    # tau = 0 (n <= leaf): K~ is K itself, so NLL/g/I are the dense formulas.
    m, t = Model(1, 48, 1, 1.5), Tree(1, 48, 1, 64)
    assert t.tau == 0
    H = hodlr.build(m, t, THETA, c=4, cap=4)
    y = np.random.default_rng(2).standard_normal(48)
    f, g, F = likelihood.evaluate(H, y)
    K = m.dense_K(THETA)
    Ks = [m.dense_K(THETA, p) for p in PARAMS]
    assert math.isclose(f, likelihood.nll(K, y), rel_tol=1e-12)
    assert np.allclose(g, likelihood.grad(K, Ks, y), rtol=1e-10)
    assert np.allclose(F, likelihood.fisher(K, Ks), rtol=1e-10)


def test_hodlr_gradient_is_derivative_of_hodlr_nll():
    m, t = Model(1, 128, 1, 1.5), Tree(1, 128, 1, 16)
    y = np.random.default_rng(4).standard_normal(128)
    H = hodlr.build(m, t, THETA, c=6, cap=6, seed=9)
    J = H.pivots()
    _, g, _ = likelihood.evaluate(H, y)
    for j in range(4):
        h = 1e-5 * THETA[j]
        tp = list(THETA); tm = list(THETA)
        tp[j] += h; tm[j] -= h
        fp = likelihood.nll(hodlr.build(m, t, tp, c=6, cap=6, seed=9, frozen=J, params=()).densify(), y)
        fm = likelihood.nll(hodlr.build(m, t, tm, c=6, cap=6, seed=9, frozen=J, params=()).densify(), y)
        assert abs((fp - fm) / (2 * h) - g[j]) <= 1e-6 * np.abs(g).max(), j


def test_fisher_scoring_reaches_the_mle():
    # well-identified two-parameter family K = s K1 + t I (K1 from the physics model)
    m = Model(1, 200, 1, 1.5)
    K1 = m.dense_K((1.0, 0.1, 5.0, 0.0))
    y = np.linalg.cholesky(2.0 * K1 + 0.3 * np.eye(200)) @ np.random.default_rng(5).standard_normal(200)

    def ev(th):
        K = th[0] * K1 + th[1] * np.eye(200)
        Ks = [K1, np.eye(200)]
        return likelihood.nll(K, y), likelihood.grad(K, Ks, y), likelihood.fisher(K, Ks)

    theta, info = scoring.fisher_scoring(ev, [1.0, 1.0], max_iter=200)
    assert info["converged"]
    res = scipy.optimize.minimize(lambda z: ev(np.exp(z))[0], np.log(theta), method="Nelder-Mead",
                                  options={"xatol": 1e-10, "fatol": 1e-13, "maxiter": 4000})
    assert info["nll"] <= res.fun + 1e-9
    assert np.allclose(theta, np.exp(res.x), rtol=1e-4)
    _, g, F = ev(theta)
    assert abs(np.linalg.solve(F, g) @ g) < 1e-10
