"""Host logic of the MLE driver and the accuracy measures (mle.py), with stand-in contexts whose
NLL, gradient and Fisher matrix are closed forms (no GPU)."""
import math

import numpy as np
import pytest

from paper_2303_10102_gb300.lib import HodlrError
from paper_2303_10102_gb300.mle import (confidence_intervals, eta_fisher, eta_score, mle_bfgs,
                                        relative_precision)


class QuadraticContext:
    """NLL(theta) = 1/2 (log theta - log t*)^T H (log theta - log t*) in log coordinates, with the
    gradient by the chain rule and the Fisher matrix J^{-1} H J^{-1} (J = diag(theta))."""

    def __init__(self, tstar, H):
        self.tstar = np.asarray(tstar, dtype=float)
        self.H = np.asarray(H, dtype=float)
        self.frozen = None
        self.calls = 0

    def _u(self, th):
        return np.log(np.asarray(th, dtype=float)) - np.log(self.tstar)

    def nll_grad(self, th, y):
        self.calls += 1
        u = self._u(th)
        return 0.5 * u @ self.H @ u, (self.H @ u) / np.asarray(th, dtype=float)

    def eval(self, th, y):
        f, g = self.nll_grad(th, y)
        Jinv = np.diag(1.0 / np.asarray(th, dtype=float))
        return f, g, Jinv @ self.H @ Jinv

    def build(self, th):
        pass

    def get_pivots(self):
        return "pivots"

    def set_pivots(self, piv):
        self.frozen = piv


def test_bfgs_reaches_the_minimum_with_badly_scaled_parameters():
    tstar = (1.3, 0.07, 8.0, 2e-3)
    A = np.array([[4.0, 1.0, 0.5, 0.0], [1.0, 3.0, 0.2, 0.1], [0.5, 0.2, 2.0, 0.3], [0.0, 0.1, 0.3, 1.0]])
    D = np.diag([1.0, 50.0, 0.2, 30.0])      # curvatures over four orders of magnitude
    H = D @ (A @ A.T) @ D
    ctx = QuadraticContext(tstar, H)
    th, info = mle_bfgs(ctx, None, (1.0, 0.1, 5.0, 1e-3), rtol=1e-10)
    assert np.allclose(th, tstar, rtol=1e-6), th
    assert info["converged"] and info["nll"] < 1e-12
    assert ctx.frozen == "pivots"          # the start point's pivot sets stay frozen afterwards
    # the returned gradient and Fisher matrix are those of the estimate
    _, g, F = ctx.eval(th, None)
    assert np.allclose(info["grad"], g) and np.allclose(info["fisher"], F)


def test_bfgs_steps_back_from_indefinite_points():
    class Fence(QuadraticContext):
        def nll_grad(self, th, y):
            if th[3] > 0.01:
                raise HodlrError(-3, "not positive definite")
            return super().nll_grad(th, y)

    ctx = Fence((1.0, 0.1, 5.0, 5e-3), np.eye(4))
    th, info = mle_bfgs(ctx, None, (2.0, 0.2, 3.0, 1e-3), rtol=1e-9)
    assert np.allclose(th, (1.0, 0.1, 5.0, 5e-3), rtol=1e-5), th

    class Broken(QuadraticContext):
        def nll_grad(self, th, y):
            raise HodlrError(-4, "non-finite")

    with pytest.raises(HodlrError):
        mle_bfgs(Broken((1, 1, 1, 1), np.eye(4)), None, (1.0, 1.0, 1.0, 1.0))


def test_intervals_and_accuracy_measures():
    F = np.array([[4.0, 1.0], [1.0, 2.0]])
    th = np.array([1.0, 2.0])
    ci, se = confidence_intervals(th, F)
    cov = np.linalg.inv(F)
    assert np.allclose(se, np.sqrt(np.diag(cov)))
    assert np.allclose(ci[:, 1] - th, 1.959963984540054 * se) and np.allclose(th - ci[:, 0], ci[:, 1] - th)
    # 90 % intervals use z = 1.6449
    ci90, _ = confidence_intervals(th, F, level=0.90)
    assert np.allclose(ci90[:, 1] - th, 1.6448536269514722 * se)
    assert relative_precision([3.0, 4.0], [3.0, 4.0]) == 0.0
    assert math.isclose(relative_precision([3.0, 4.0], [0.0, 0.0 + 5.0]), math.hypot(3.0, 1.0) / 5.0)
    # eta_score: the I^{-1} norm; with I = diag(4, 1) the difference (2, 1) has norm sqrt(1 + 1)
    assert math.isclose(eta_score([2.0, 1.0], [0.0, 0.0], np.diag([4.0, 1.0])), math.sqrt(2.0))
    # eta_fisher: zero for equal matrices; for scalars tr((a - b)(1/a - 1/b)) = -(a - b)^2 / (a b)
    assert eta_fisher(F, F) == 0.0
    a, b = 4.0, 2.0
    assert math.isclose(eta_fisher([[b]], [[a]]), math.sqrt((a - b) ** 2 / (a * b)))
