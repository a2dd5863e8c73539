"""The seeded input recipe: synth.simulate_y draws y ~ N(0, K(theta)) for the model the estimator
fits (circulant-embedding Matern field through the physics map, plus tau2 noise).

Checked on CPU against the oracle's dense K (explicit matrices, eq. cov model) with many seeds:
the sample covariance must agree with K within its sampling error, and the whitened sample
covariance must have unit mean eigenvalue (this checks the small tau2 directions too)."""
import numpy as np
import pytest

import synth
from oracle.physics import Model

CASES = [
    dict(dim=1, G=32, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-3)),
    dict(dim=1, G=16, nvar=2, nu=0.5, theta=(1.3, 0.07, 8.0, 2e-3)),
    dict(dim=2, G=8, nvar=1, nu=0.5, theta=(1.0, 0.1, 8.0, 1e-3)),
]


@pytest.mark.parametrize("case", CASES, ids=["1d-uni", "1d-biv", "2d-uni"])
def test_simulated_data_has_the_model_covariance(case):
    w = synth.small_workload(dim=case["dim"], G=case["G"], nvar=case["nvar"], nu=case["nu"], theta=case["theta"])
    K = Model(w.dim, w.G, w.nvar, w.nu).dense_K(w.theta)
    N = K.shape[0]
    n = 20000
    Y = np.stack([synth.simulate_y(w, seed=1000 + s) for s in range(n)])
    assert Y.shape == (n, N)
    C = Y.T @ Y / n
    # sampling error of a Gaussian sample covariance: E||C - K||_F^2 = (||K||_F^2 + tr(K)^2) / n
    rms = np.sqrt((np.sum(K * K) + np.trace(K) ** 2) / n)
    assert np.linalg.norm(C - K) <= 4.0 * rms, (np.linalg.norm(C - K), rms)
    # whitened: W = L^{-1} C L^{-T} ~ I, tr(W)/N = 1 +- sqrt(2 / (n N))
    L = np.linalg.cholesky(K)
    Z = np.linalg.solve(L, Y.T)
    mean_eig = np.sum(Z * Z) / (n * N)
    assert abs(mean_eig - 1.0) <= 5.0 * np.sqrt(2.0 / (n * N)), mean_eig
