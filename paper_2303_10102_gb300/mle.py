"""Maximum-likelihood estimation and uncertainty quantification on the HODLR likelihood (host
logic over the CUDA evaluation of include/hodlr.h).

* ``mle_bfgs``: quasi-Newton (BFGS) minimisation of the NLL of K~(theta) over log theta (the
  parameters stay positive), with the library's exact gradient (Sec. 2.2: the MLE is found by
  a quasi-Newton method on the approximated likelihood; the paper's optimiser stops at a
  relative tolerance of 1e-6, Sec. 5.2.3).  The probes are fixed by the context's seed and the
  pivot sets of the rank decisions are frozen at the start point, so the objective is a smooth
  function of theta (Sec. 3.3 keeps the sampling pattern fixed).
* ``confidence_intervals``: asymptotic intervals theta^ +- z sqrt(diag(I(theta^)^{-1})) from the
  expected Fisher information at the estimate (Sec. 2.2, eq. CLT and eq. fisher info).
* ``relative_precision`` / ``eta_score`` / ``eta_fisher``: the accuracy measures of Sec. 5.2.2
  (relative precision of the log-likelihood, score and Fisher matrix, and the scale-free errors
  of eq. score-error and eq. fisher-error), for comparing the HODLR values with exact ones.
"""
from __future__ import annotations

import math

import numpy as np

from .lib import HodlrError


def mle_bfgs(ctx, y, theta0, rtol=1e-6, max_iter=200, freeze_pivots=True, history=None):
    """Minimise NLL~(theta) from theta0 by BFGS.

    The variables are whitened log-parameters u = C^T (log theta - log theta0), with C C^T the
    Fisher information in log coordinates at theta0 (J I(theta0) J, J = diag(theta0)), so that the
    Hessian of the NLL in u is close to the identity: the four parameters differ by orders of
    magnitude in scale and curvature.  Returns (theta_hat, info) with info = {"nll", "grad",
    "fisher", "iterations", "converged", "message"}, the gradient and Fisher matrix evaluated at
    theta_hat.  With freeze_pivots the context keeps the start point's pivot sets afterwards (call
    ctx.set_pivots(None) to release them).  Points where K~ is not positive definite
    (HODLR_ENOTPD) count as +inf, which makes the line search step back."""
    from scipy.optimize import minimize

    theta0 = np.asarray(theta0, dtype=np.float64)
    if freeze_pivots:
        ctx.build(theta0)
        ctx.set_pivots(ctx.get_pivots())
    _, _, F0 = ctx.eval(theta0, y)
    J = np.diag(theta0)
    C = np.linalg.cholesky(J @ np.asarray(F0) @ J)       # log coordinates, whitened
    Cinv_T = np.linalg.inv(C).T
    cache = {}

    def theta_of(u):
        return theta0 * np.exp(Cinv_T @ u)

    def fun(u):
        th = theta_of(u)
        key = tuple(th)
        if key not in cache:
            try:
                f, g = ctx.nll_grad(th, y)
            except HodlrError as e:
                if e.code != -3:
                    raise
                cache[key] = (np.inf, np.zeros(4))
            else:
                # d/du = C^{-1} (theta * d/dtheta)
                cache[key] = (f, np.linalg.solve(C, np.asarray(g) * th))
            if history is not None:
                history.append({"theta": th.tolist(), "nll": cache[key][0]})
        return cache[key]

    # in whitened coordinates a unit step is one standard error: stop when the gradient is below
    # rtol of that scale or the relative step is below rtol
    res = minimize(fun, np.zeros(4), jac=True, method="BFGS",
                   options={"gtol": rtol, "xrtol": rtol, "maxiter": max_iter})
    theta = theta_of(res.x)
    f, g, F = ctx.eval(theta, y)
    return theta, {"nll": float(f), "grad": np.asarray(g).tolist(), "fisher": np.asarray(F).tolist(),
                   "iterations": int(res.nit), "converged": bool(res.success), "message": str(res.message)}


def confidence_intervals(theta_hat, fisher, level=0.95):
    """Asymptotic intervals theta^_j +- z_{(1+level)/2} sqrt((I^{-1})_jj) (eq. CLT)."""
    from scipy.stats import norm

    cov = np.linalg.inv(np.asarray(fisher, dtype=np.float64))
    z = norm.ppf(0.5 * (1.0 + level))
    se = np.sqrt(np.diag(cov))
    th = np.asarray(theta_hat, dtype=np.float64)
    return np.stack([th - z * se, th + z * se], axis=1), se


def relative_precision(approx, exact):
    """Relative precision ||approx - exact|| / ||exact|| (Frobenius / 2-norm / absolute value)."""
    a, e = np.asarray(approx, dtype=np.float64), np.asarray(exact, dtype=np.float64)
    return float(np.linalg.norm(a - e) / max(np.linalg.norm(e), 1e-300))


def eta_score(score, score_exact, fisher_exact):
    """||S - S~|| in the I^{-1} norm (eq. score-error)."""
    d = np.asarray(score, dtype=np.float64) - np.asarray(score_exact, dtype=np.float64)
    return float(math.sqrt(abs(d @ np.linalg.solve(np.asarray(fisher_exact, dtype=np.float64), d))))


def eta_fisher(fisher, fisher_exact):
    """tr((I - I~)(I^{-1} - I~^{-1}))^{1/2} (eq. fisher-error)."""
    F = np.asarray(fisher, dtype=np.float64)
    F0 = np.asarray(fisher_exact, dtype=np.float64)
    return float(math.sqrt(abs(np.trace((F0 - F) @ (np.linalg.inv(F0) - np.linalg.inv(F))))))
