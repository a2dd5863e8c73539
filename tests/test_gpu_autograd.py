"""The differentiable NLL on the GPU: autograd's theta-gradient (reverse mode through the
factorization) equals the trace-route score of the library, the oracle's score and central
differences of the GPU NLL; the y-gradient equals K~^{-1} y of the densified oracle K~."""
import numpy as np
import pytest
import torch

import synth
from oracle import hodlr as oh, likelihood as ol
from oracle.physics import Model
from oracle.tree import Tree

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_autograd_matches_score_and_oracle():
    from paper_2303_10102_gb300 import Hodlr
    from paper_2303_10102_gb300.autograd import hodlr_nll
    w = synth.small_workload(dim=1, G=512, nvar=1, nu=1.5, theta=(1.0, 0.1, 5.0, 1e-3), leaf=32, cap=10, c=12)
    m, t = Model(1, w.G, 1, 1.5), Tree(1, w.G, 1, 32)
    y_np = synth.simulate_y(w)
    h = Hodlr(1, w.G, 1, 1.5, "fp64", 32, 10, 2, 0.0, 1, device=DEV, guard=1e-5)
    theta = torch.tensor(w.theta, dtype=torch.float64, requires_grad=True)
    y = torch.as_tensor(y_np, device=DEV).requires_grad_(True)
    loss = hodlr_nll(h, theta, y)
    loss.backward()
    g_lib = h.grad(w.theta, y.detach())                 # forward (tangent) mode, exact traces
    assert np.array_equal(theta.grad.numpy(), h.grad_adjoint(w.theta, y.detach()))
    assert np.all(np.abs(theta.grad.numpy() - g_lib) <= 1e-9 * np.abs(g_lib).max())
    # central differences of the GPU NLL (probes and pivot sets frozen: Sec. 3.3)
    h.build(w.theta)
    h.set_pivots(h.get_pivots())
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1e-5 * w.theta[j]
        fd = (h.nll(np.asarray(w.theta) + e, y.detach()) - h.nll(np.asarray(w.theta) - e, y.detach())) / (2 * e[j])
        assert abs(fd - theta.grad.numpy()[j]) <= 1e-6 * np.abs(theta.grad.numpy()).max(), (j, fd, theta.grad)
    h.set_pivots(None)
    H = oh.build(m, t, w.theta, c=12, cap=10, guard=1e-5, seed=1)
    f0, g0, _ = ol.evaluate(H, t.to_tree(y_np))
    assert abs(loss.item() - f0) <= 1e-10 * abs(f0)
    assert np.abs(theta.grad.numpy() - g0).max() <= 1e-8 * np.abs(g0).max()
    # y-gradient: alpha = K~^{-1} y (tree order in the oracle, natural order here)
    alpha = np.linalg.solve(H.densify(), t.to_tree(y_np))
    a_nat = np.empty_like(alpha)
    a_nat[t.perm] = alpha
    gy = y.grad.detach().cpu().numpy()
    assert np.abs(gy - a_nat).max() <= 1e-9 * np.abs(a_nat).max()
