"""Reverse mode through the factorization (hodlr_grad_adjoint) against the forward route.

The adjoint route assembles the score from Kbar = (K~^{-1} - alpha alpha^T) / 2 pulled back onto
the HODLR factors and contracted with Alg. 2's tangent factors; the forward route takes the exact
traces of App. B.  Both are the derivative of the same NLL~(theta), so they agree to rounding:
on every small FP64 case (1-D and 2-D, univariate and bivariate, uneven trees) within 1e-9 of the
largest component, and against the FP64 oracle's score within its gradient tolerance; on the
mixed BF16 path at C2's settings (P2) within 1e-6.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import likelihood as ol

from test_gpu_parity import GRAD_TOL, SMALL, ctx, oracle_build

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("name", list(SMALL))
def test_adjoint_gradient_equals_trace_route_fp64(name):
    w = SMALL[name]
    y = synth.simulate_y(w)
    h = ctx(w, "fp64")
    yd = torch.as_tensor(y, device=DEV)
    g = np.asarray(h.grad(w.theta, yd))
    ga = np.asarray(h.grad_adjoint(w.theta, yd))
    assert np.all(np.abs(ga - g) <= 1e-9 * np.abs(g).max()), (ga, g)
    m, t, H = oracle_build(w, "fp64")
    _, g0, _ = ol.evaluate(H, t.to_tree(y))
    assert np.abs(ga - g0).max() <= GRAD_TOL.get(name, 1e-9) * np.abs(g0).max(), (ga, g0)


def test_adjoint_gradient_mixed_bf16_p2():
    w = synth.workload("P2")
    from paper_2303_10102_gb300 import Hodlr
    h = Hodlr(w.dim, w.G, w.nvar, w.nu, "bf16", w.leaf, w.cap, w.c - w.cap, w.tol, w.seed_probe, device=DEV,
              guard=w.guard)
    yd = torch.as_tensor(synth.simulate_y(w), device=DEV)
    g = np.asarray(h.grad(w.theta, yd))
    ga = np.asarray(h.grad_adjoint(w.theta, yd))
    print(f"P2 bf16: adjoint vs trace route, max |diff| / max |g| = {np.abs(ga - g).max() / np.abs(g).max():.2e}")
    assert np.all(np.abs(ga - g) <= 1e-6 * np.abs(g).max()), (ga, g)
