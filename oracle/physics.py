"""Physics-based covariance K(theta) and its derivatives (oracle).

Model (Sec. 2.1, eq. cov model, exact because the map is linear):
    univariate   K = A^{-1} K_u A^{-T} + tau2 I                      (y = A^{-1} u)
    bivariate    K = L K_u L^T + tau2 I,  L = [I; A^{-1}]            (y = (u, A^{-1} u))
with A = -Laplacian_h + kappa^2 I (3-point / 5-point finite differences, Dirichlet,
interior nodes x_i = i h, h = 1/(G+1)) and K_u = sigma2 * M_{nu,ell} the Matern
covariance of eq. whittle covariance (Sec. 5.1):
    M(r) = (2^{nu-1} Gamma(nu))^{-1} (r/ell)^nu K_nu(r/ell),
which is exp(-r/ell) for nu = 1/2 and (1 + r/ell) exp(-r/ell) for nu = 3/2
(the paper's convention: no sqrt(2 nu) factor).

theta = (sigma2, ell, kappa, tau2).  K is only accessed through products K X
(Sec. 3.2: "assume there exists a fast solver of computing matrix-vector products"):
A^{-1} by a banded solve (1-D) or an orthonormal DST-I diagonalisation (2-D), and
K_u by zero-padded FFT circulant embedding of the Toeplitz / block-Toeplitz matrix,
which is an exact product.  Derivatives follow by differentiating the product
(Sec. 3.3: K_j S = d(K S)/d theta_j):
    dA^{-1}/dkappa = -2 kappa A^{-2},  dK_u/dell = sigma2 dM/dell,  dK/dsigma2 = (K - tau2 I)/sigma2,
    dK/dtau2 = I.
Vectors are in natural layout (bivariate: [x1 (Ns); x2 (Ns)]); the 2-D natural
index is iy * G + ix.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg

PARAMS = ("sigma2", "ell", "kappa", "tau2")


def matern(r, ell, nu):
    """M_{nu,ell}(r) of eq. whittle covariance for nu in {1/2, 3/2}."""
    z = np.asarray(r, dtype=np.float64) / ell
    if nu == 0.5:
        return np.exp(-z)
    if nu == 1.5:
        return (1.0 + z) * np.exp(-z)
    raise ValueError("nu must be 0.5 or 1.5")


def matern_dell(r, ell, nu):
    """d M_{nu,ell}(r) / d ell."""
    z = np.asarray(r, dtype=np.float64) / ell
    if nu == 0.5:
        return (z / ell) * np.exp(-z)
    if nu == 1.5:
        return (z * z / ell) * np.exp(-z)
    raise ValueError("nu must be 0.5 or 1.5")


class Model:
    """Grid, physics operator and latent covariance of one workload."""

    def __init__(self, dim: int, G: int, nvar: int, nu: float):
        self.dim, self.G, self.nvar, self.nu = dim, G, nvar, nu
        self.h = 1.0 / (G + 1)
        self.Ns = G ** dim
        self.N = nvar * self.Ns

    # ---------------------------------------------------------------- A^{-1}
    def solve_A(self, X, kappa):
        """A^{-1} X for X of shape (Ns, q)."""
        G, h = self.G, self.h
        X = np.asarray(X, dtype=np.float64)
        if self.dim == 1:
            ab = np.zeros((3, G))
            ab[0, 1:] = -1.0 / h ** 2
            ab[1, :] = 2.0 / h ** 2 + kappa ** 2
            ab[2, :-1] = -1.0 / h ** 2
            return scipy.linalg.solve_banded((1, 1), ab, X)
        q = X.shape[1]
        j = np.arange(1, G + 1)
        lam = 4.0 * np.sin(j * np.pi / (2.0 * (G + 1))) ** 2 / h ** 2   # eigenvalues of 1-D -D2
        F = X.reshape(G, G, q)                                            # [iy, ix, col]
        F = scipy.fft.dst(F, type=1, norm="ortho", axis=0)
        F = scipy.fft.dst(F, type=1, norm="ortho", axis=1)
        F = F / (lam[:, None, None] + lam[None, :, None] + kappa ** 2)
        F = scipy.fft.idst(F, type=1, norm="ortho", axis=1)
        F = scipy.fft.idst(F, type=1, norm="ortho", axis=0)
        return F.reshape(G * G, q)

    # ---------------------------------------------------------------- K_u
    def _embedding(self, sigma2, ell, which):
        G, h = self.G, self.h
        L = 2 * G
        k = np.arange(L)
        d = np.minimum(k, L - k).astype(np.float64)
        f = matern if which == "K" else matern_dell
        if self.dim == 1:
            return sigma2 * f(h * d, ell, self.nu)
        dx, dy = np.meshgrid(d, d, indexing="xy")
        return sigma2 * f(h * np.sqrt(dx * dx + dy * dy), ell, self.nu)

    def apply_Ku(self, X, sigma2, ell, which="K"):
        """K_u X (which="K") or (dK_u/dell) X (which="ell") by circulant embedding."""
        G = self.G
        X = np.asarray(X, dtype=np.float64)
        q = X.shape[1]
        emb = self._embedding(sigma2, ell, which)
        if self.dim == 1:
            lam = np.fft.rfft(emb)
            P = np.zeros((2 * G, q))
            P[:G] = X
            Y = np.fft.irfft(lam[:, None] * np.fft.rfft(P, axis=0), n=2 * G, axis=0)
            return Y[:G]
        lam = np.fft.rfft2(emb)
        P = np.zeros((2 * G, 2 * G, q))
        P[:G, :G] = X.reshape(G, G, q)
        Y = np.fft.irfft2(lam[:, :, None] * np.fft.rfft2(P, axes=(0, 1)), s=(2 * G, 2 * G), axes=(0, 1))
        return Y[:G, :G].reshape(G * G, q)

    # ---------------------------------------------------------------- K, K_j
    def apply(self, X, theta, which="K"):
        """K X or (dK/dtheta_j) X; X has shape (N, q) in natural layout."""
        sigma2, ell, kappa, tau2 = theta
        X = np.asarray(X, dtype=np.float64)
        if X.ndim == 1:
            return self.apply(X[:, None], theta, which)[:, 0]
        if which == "tau2":
            return X.copy()
        if which == "sigma2":
            return (self.apply(X, theta, "K") - tau2 * X) / sigma2
        Ns = self.Ns
        sA = lambda V: self.solve_A(V, kappa)
        if self.nvar == 1:
            if which == "K":
                return sA(self.apply_Ku(sA(X), sigma2, ell)) + tau2 * X
            if which == "ell":
                return sA(self.apply_Ku(sA(X), sigma2, ell, "ell"))
            if which == "kappa":
                # d/dkappa [A^{-1} K_u A^{-1}] with dA^{-1}/dkappa = -2 kappa A^{-2}
                t1 = sA(sA(self.apply_Ku(sA(X), sigma2, ell)))
                t2 = sA(self.apply_Ku(sA(sA(X)), sigma2, ell))
                return -2.0 * kappa * (t1 + t2)
            raise ValueError(which)
        x1, x2 = X[:Ns], X[Ns:]
        w = x1 + sA(x2)                                          # L^T x
        if which == "K":
            u = self.apply_Ku(w, sigma2, ell)
            return np.concatenate([u, sA(u)]) + tau2 * X
        if which == "ell":
            u = self.apply_Ku(w, sigma2, ell, "ell")
            return np.concatenate([u, sA(u)])
        if which == "kappa":
            # dL/dkappa = [0; -2 kappa A^{-2}]:  dL K_u L^T x + L K_u dL^T x
            u = self.apply_Ku(w, sigma2, ell)
            s = self.apply_Ku(-2.0 * kappa * sA(sA(x2)), sigma2, ell)
            return np.concatenate([s, sA(s) - 2.0 * kappa * sA(sA(u))])
        raise ValueError(which)

    # ---------------------------------------------------------------- dense (small grids)
    def points(self):
        x = self.h * np.arange(1, self.G + 1)
        if self.dim == 1:
            return x[:, None]
        iy, ix = np.divmod(np.arange(self.Ns), self.G)
        return np.stack([x[ix], x[iy]], axis=1)

    def dense_A(self, kappa):
        G, h = self.G, self.h
        T = (np.diag(np.full(G, 2.0)) - np.diag(np.ones(G - 1), 1) - np.diag(np.ones(G - 1), -1)) / h ** 2
        if self.dim == 1:
            return T + kappa ** 2 * np.eye(G)
        I = np.eye(G)
        return np.kron(I, T) + np.kron(T, I) + kappa ** 2 * np.eye(G * G)

    def dense_Ku(self, sigma2, ell, which="K"):
        P = self.points()
        r = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
        f = matern if which == "K" else matern_dell
        return sigma2 * f(r, ell, self.nu)

    def dense_K(self, theta, which="K"):
        """Dense K or dK/dtheta_j from explicit matrices (small grids only)."""
        sigma2, ell, kappa, tau2 = theta
        Ai = np.linalg.inv(self.dense_A(kappa))
        dAi = -2.0 * kappa * Ai @ Ai
        Ku = self.dense_Ku(sigma2, ell)
        Ns = self.Ns
        if self.nvar == 1:
            Lm, dLm = Ai, dAi
        else:
            Lm = np.vstack([np.eye(Ns), Ai])
            dLm = np.vstack([np.zeros((Ns, Ns)), dAi])
        if which == "K":
            return Lm @ Ku @ Lm.T + tau2 * np.eye(self.N)
        if which == "sigma2":
            return Lm @ (Ku / sigma2) @ Lm.T
        if which == "ell":
            return Lm @ self.dense_Ku(sigma2, ell, "ell") @ Lm.T
        if which == "kappa":
            return dLm @ Ku @ Lm.T + Lm @ Ku @ dLm.T
        if which == "tau2":
            return np.eye(self.N)
        raise ValueError(which)
