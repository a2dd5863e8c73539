"""Fisher-scoring outer loop (oracle).

The paper maximises the likelihood with a quasi-Newton method and uses the Fisher
information for confidence intervals (Sec. 2.2, eq. CLT; Sec. 5.2.3).  The large 2-D
workload iterates Fisher scoring instead:
    theta <- theta - I(theta)^{-1} g(theta)      (g = dNLL/dtheta = -S)
until ||dtheta||_2 / ||theta||_2 < rtol (1e-6, mirroring the paper's relative
tolerance), halving the step while the NLL rises or theta leaves the positive orthant.
`evaluate(theta)` returns (nll, g, I) and is supplied by the caller.
"""
from __future__ import annotations

import numpy as np


def fisher_scoring(evaluate, theta0, rtol=1e-6, max_iter=50, max_halvings=30, history=None):
    theta = np.asarray(theta0, dtype=np.float64).copy()
    f, g, F = evaluate(theta)
    for it in range(max_iter):
        step = -np.linalg.solve(F, g)
        t = 1.0
        for _ in range(max_halvings):
            cand = theta + t * step
            if np.all(cand > 0.0):
                fc, gc, Fc = evaluate(cand)
                if np.isfinite(fc) and fc <= f + 1e-12 * abs(f):
                    break
            t *= 0.5
        else:
            return theta, {"iterations": it, "converged": False, "nll": f}
        dtheta = cand - theta
        theta, f, g, F = cand, fc, gc, Fc
        if history is not None:
            history.append({"theta": theta.tolist(), "nll": f})
        if np.linalg.norm(dtheta) / np.linalg.norm(theta) < rtol:
            return theta, {"iterations": it + 1, "converged": True, "nll": f}
    return theta, {"iterations": max_iter, "converged": False, "nll": f}
