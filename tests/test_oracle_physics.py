"""Pins of the oracle's physics products K X and K_j X (eq. cov model; eq. whittle covariance)."""
import numpy as np
import pytest
import scipy.special

from oracle.physics import Model, matern, matern_dell

THETA = (1.3, 0.12, 6.0, 2e-3)


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_matern_matches_bessel_form(nu):
    # eq. whittle covariance with K_nu from scipy
    ell = 0.07
    r = np.linspace(1e-3, 0.5, 50)
    z = r / ell
    ref = z ** nu * scipy.special.kv(nu, z) / (2 ** (nu - 1) * scipy.special.gamma(nu))
    assert np.allclose(matern(r, ell, nu), ref, rtol=1e-12, atol=0)
    assert matern(0.0, ell, nu) == 1.0
    h = 1e-6
    fd = (matern(r, ell + h, nu) - matern(r, ell - h, nu)) / (2 * h)
    assert np.allclose(matern_dell(r, ell, nu), fd, rtol=1e-6, atol=1e-12)


def test_dst_eigenvalues_closed_form():
    m = Model(1, 50, 1, 1.5)
    ev = np.linalg.eigvalsh(m.dense_A(3.0))
    j = np.arange(1, 51)
    ref = 4.0 / m.h ** 2 * np.sin(j * np.pi * m.h / 2) ** 2 + 9.0
    assert np.allclose(ev, np.sort(ref), rtol=1e-12)


CASES = [(1, 64, 1, 1.5), (1, 48, 2, 0.5), (2, 8, 1, 0.5), (2, 6, 2, 1.5)]


@pytest.mark.parametrize("dim,G,nvar,nu", CASES)
@pytest.mark.parametrize("which", ["K", "sigma2", "ell", "kappa", "tau2"])
def test_apply_matches_dense(dim, G, nvar, nu, which):
    m = Model(dim, G, nvar, nu)
    X = np.random.default_rng(0).standard_normal((m.N, 3))
    D = m.dense_K(THETA, which)
    Y = m.apply(X, THETA, which)
    assert np.abs(Y - D @ X).max() <= 1e-12 * np.abs(D @ X).max()


@pytest.mark.parametrize("dim,G,nvar,nu", CASES)
def test_dense_derivatives_are_derivatives(dim, G, nvar, nu):
    m = Model(dim, G, nvar, nu)
    for j, which in enumerate(["sigma2", "ell", "kappa", "tau2"]):
        h = 1e-5 * THETA[j]
        tp = list(THETA); tm = list(THETA)
        tp[j] += h; tm[j] -= h
        fd = (m.dense_K(tp) - m.dense_K(tm)) / (2 * h)
        an = m.dense_K(THETA, which)
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max()


def test_model_symmetric_positive_definite():
    m = Model(2, 6, 2, 1.5)
    K = m.dense_K(THETA)
    assert np.allclose(K, K.T, rtol=0, atol=1e-12 * np.abs(K).max())
    assert np.linalg.eigvalsh(K).min() > 0
