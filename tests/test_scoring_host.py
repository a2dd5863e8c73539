"""Host logic of the Fisher-scoring loop (Sec. 2.2; stopping rule of Sec. 5.2.3) with stand-in
contexts whose NLL, score and Fisher information are closed forms (no GPU):
  * on a quadratic NLL the first step is the exact Newton step to the minimiser, and the loop
    then stops on ||dtheta|| / ||theta|| < rtol;
  * candidates outside the positive orthant, candidates that make K~ indefinite (ENOTPD) and
    candidates that raise the NLL are halved away;
  * other library errors propagate."""
import numpy as np
import pytest

from paper_2303_10102_gb300.lib import HodlrError
from paper_2303_10102_gb300.scoring import fisher_scoring


class Quadratic:
    """NLL = 1/2 (theta - t*)^T A (theta - t*), score A (theta - t*), Fisher A."""

    def __init__(self, tstar, A, enotpd_if=None, other_error_if=None):
        self.tstar = np.asarray(tstar, dtype=np.float64)
        self.A = np.asarray(A, dtype=np.float64)
        self.enotpd_if = enotpd_if
        self.other_error_if = other_error_if
        self.evaluated = []

    def eval(self, theta, y):
        theta = np.asarray(theta, dtype=np.float64)
        self.evaluated.append(theta.copy())
        if self.other_error_if is not None and self.other_error_if(theta):
            raise HodlrError(-4, "non-finite")
        if self.enotpd_if is not None and self.enotpd_if(theta):
            raise HodlrError(-3, "not SPD")
        d = theta - self.tstar
        return 0.5 * d @ self.A @ d, self.A @ d, self.A.copy()


A4 = np.diag([2.0, 5.0, 1.0, 3.0]) + 0.1


def test_newton_step_then_stop():
    q = Quadratic([1.0, 0.1, 8.0, 1e-3], A4)
    hist = []
    theta, info = fisher_scoring(q, None, [1.5, 0.2, 6.0, 2e-3], history=hist)
    assert info["converged"]
    np.testing.assert_allclose(hist[0]["theta"], q.tstar, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(theta, q.tstar, rtol=1e-12, atol=1e-15)
    assert info["iterations"] == 2   # the second step is zero to rounding


def test_halving_keeps_the_positive_orthant():
    # the full step lands at a negative tau2; halving keeps every candidate accepted positive
    q = Quadratic([1.0, 0.1, 8.0, -1.0], A4)
    hist = []
    fisher_scoring(q, None, [1.0, 0.1, 8.0, 0.5], max_iter=5, history=hist)
    assert hist and all(min(h["theta"]) > 0.0 for h in hist)
    assert all(min(t) > 0.0 for t in q.evaluated)


def test_enotpd_candidates_are_halved_away():
    q = Quadratic([2.0, 0.1, 8.0, 1e-3], np.eye(4), enotpd_if=lambda th: th[0] > 1.6)
    hist = []
    fisher_scoring(q, None, [1.0, 0.1, 8.0, 1e-3], max_iter=1, history=hist)
    # full step to 2.0 and half step to 1.5 + ... : the first accepted candidate has theta_0 <= 1.6
    assert hist[0]["theta"][0] == pytest.approx(1.5)
    assert any(t[0] > 1.6 for t in q.evaluated)


def test_other_errors_propagate():
    q = Quadratic([2.0, 0.1, 8.0, 1e-3], np.eye(4), other_error_if=lambda th: th[0] > 1.6)
    with pytest.raises(HodlrError) as e:
        fisher_scoring(q, None, [1.0, 0.1, 8.0, 1e-3], max_iter=1)
    assert e.value.code == -4


def test_no_descent_stops_without_moving():
    class Flat(Quadratic):
        def eval(self, theta, y):
            f, g, F = super().eval(theta, y)
            return f if np.allclose(theta, [1.0, 0.1, 8.0, 1e-3]) else f + 1.0, g, F
    q = Flat([2.0, 0.1, 8.0, 1e-3], np.eye(4))
    theta, info = fisher_scoring(q, None, [1.0, 0.1, 8.0, 1e-3], max_iter=3, max_halvings=4)
    assert not info["converged"] and info["iterations"] == 0
    np.testing.assert_array_equal(theta, [1.0, 0.1, 8.0, 1e-3])
