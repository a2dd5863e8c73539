"""Fisher scoring on the HODLR likelihood (host loop over hodlr_eval).

Each iteration evaluates NLL, gradient g and expected Fisher information I of the HODLR
approximation at theta (one call into the CUDA library) and moves
theta <- theta - t I^{-1} g, halving t while the candidate leaves the positive orthant,
makes K~ indefinite (the library reports ENOTPD) or raises the NLL; it stops when
||dtheta||_2 / ||theta||_2 < rtol.  The Fisher information is the expected information of
eq. fisher info approximated (Sec. 4.3); the 1e-6 relative tolerance follows the paper's
optimiser setting (Sec. 5.2.3).
"""
from __future__ import annotations

import numpy as np

from .lib import HodlrError


def fisher_scoring(ctx, y, theta0, rtol=1e-6, max_iter=50, max_halvings=30, history=None):
    theta = np.asarray(theta0, dtype=np.float64).copy()
    f, g, F = ctx.eval(theta, y)
    for it in range(max_iter):
        step = -np.linalg.solve(F, g)
        t = 1.0
        cand = None
        for _ in range(max_halvings):
            c = theta + t * step
            if np.all(c > 0.0):
                try:
                    fc, gc, Fc = ctx.eval(c, y)
                except HodlrError as e:
                    if e.code != -3:
                        raise
                    fc = np.inf
                if np.isfinite(fc) and fc <= f + 1e-12 * abs(f):
                    cand = c
                    break
            t *= 0.5
        if cand is None:
            return theta, {"iterations": it, "converged": False, "nll": f}
        dtheta = cand - theta
        theta, f, g, F = cand, fc, gc, Fc
        if history is not None:
            history.append({"theta": theta.tolist(), "nll": f})
        if np.linalg.norm(dtheta) / np.linalg.norm(theta) < rtol:
            return theta, {"iterations": it + 1, "converged": True, "nll": f}
    return theta, {"iterations": max_iter, "converged": False, "nll": f}
