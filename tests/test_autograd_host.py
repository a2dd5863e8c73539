"""Host logic of the autograd wrapper (no GPU): forward evaluates the NLL only; the backward
pass asks the library for the reverse-mode gradient at the forward theta, scaled by the incoming
gradient, and for K~^{-1} y for the data, from a stand-in context whose values are fixed."""
import numpy as np
import torch

from paper_2303_10102_gb300.autograd import hodlr_nll


class FakeContext:
    """Stands in for lib.Hodlr: NLL = 1/2 y^T D^{-1} y + c with a diagonal D and a fixed score."""

    def __init__(self, d):
        self.d = torch.as_tensor(d, dtype=torch.float64)
        self.calls = []

    def nll(self, theta, y):
        self.calls.append(("nll", tuple(theta)))
        return float(0.5 * (y * y / self.d).sum() + 3.0)

    def grad_adjoint(self, theta, y):
        self.calls.append(("grad_adjoint", tuple(theta)))
        return np.array([1.0, -2.0, 0.5, 4.0])

    def solve(self, y):
        self.calls.append(("solve",))
        return y / self.d


def test_backward_theta_and_y():
    h = FakeContext([1.0, 2.0, 4.0])
    theta = torch.tensor([1.0, 0.1, 5.0, 1e-4], dtype=torch.float64, requires_grad=True)
    y = torch.tensor([1.0, -1.0, 2.0], dtype=torch.float64, requires_grad=True)
    loss = 2.0 * hodlr_nll(h, theta, y)
    loss.backward()
    assert torch.equal(theta.grad, torch.tensor([2.0, -4.0, 1.0, 8.0], dtype=torch.float64))
    assert torch.allclose(y.grad, 2.0 * y.detach() / h.d)
    th = (1.0, 0.1, 5.0, 1e-4)
    # forward: NLL only; backward: the adjoint gradient at the forward theta, then K~^{-1} y
    assert h.calls[0] == ("nll", th) and h.calls[1] == ("grad_adjoint", th)
    assert h.calls[2] == ("nll", th) and h.calls[3] == ("solve",)


def test_no_solve_without_y_grad():
    h = FakeContext([1.0, 1.0])
    theta = torch.tensor([1.0, 0.1, 5.0, 1e-4], dtype=torch.float64, requires_grad=True)
    y = torch.tensor([0.5, 0.25], dtype=torch.float64)
    hodlr_nll(h, theta, y).backward()
    assert [c[0] for c in h.calls] == ["nll", "grad_adjoint"]
    assert theta.grad is not None
