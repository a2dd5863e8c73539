"""The approximate negative log-likelihood as a differentiable PyTorch function.

The paper states that the HODLR construction can be differentiated (Sec. 3.3) and computes
the score from the derivative matrices K~_j of Alg. 2 with exact traces (Sec. 4.3,
App. B).  ``hodlr_nll`` exposes the likelihood to autograd with a reverse-mode backward:

* forward: L(theta) = N/2 log 2 pi + 1/2 log det K~ + 1/2 y^T K~^{-1} y (eq. log-like
  approximated): one build (with Alg. 2's tangent factors) and one factorization through the
  C ABI;
* backward with respect to theta: the adjoint of L with respect to K~, Kbar = (K~^{-1} -
  alpha alpha^T) / 2, pulled back through the factorization onto the HODLR factors and
  contracted with their tangents (hodlr_grad_adjoint): the same score as the trace route of
  eq. score approximated, by the other mode;
* backward with respect to y: dL/dy = K~^{-1} y, one more solve with the stored factors.

Nothing here computes on the host: every value comes from the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch


class _HodlrNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, y, h):
        th = theta.detach().to("cpu", torch.float64).numpy()
        nll = h.nll(th, y.detach())
        ctx.h, ctx.th = h, th
        ctx.save_for_backward(y)
        return torch.tensor(nll, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (y,) = ctx.saved_tensors
        g_theta = g_y = None
        if ctx.needs_input_grad[0]:
            # reverse mode through the factorization, on the build of the forward call (rebuilt
            # only if the context was used at another theta in between)
            grad = ctx.h.grad_adjoint(ctx.th, y.detach())
            g_theta = gout.to(torch.float64) * torch.as_tensor(np.asarray(grad, dtype=np.float64))
        if ctx.needs_input_grad[1]:
            # K~^{-1} y with the factors of this theta: the evaluation rebuilds only if the
            # context was used at another theta in between
            ctx.h.nll(ctx.th, y.detach())
            alpha = ctx.h.solve(y.detach())
            g_y = (gout.to(alpha.device, torch.float64) * alpha).to(y.dtype)
        return g_theta, g_y, None


def hodlr_nll(h, theta: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Differentiable NLL of context ``h`` (a ``lib.Hodlr``) at ``theta`` (4 values, any device)
    for data ``y`` (N values on the context's device, natural order).  Returns a 0-d FP64 CPU
    tensor; ``.backward()`` fills ``theta.grad`` (CPU) and ``y.grad`` (device)."""
    if theta.numel() != 4:
        raise ValueError("theta must hold (sigma2, ell, kappa, tau2)")
    return _HodlrNLL.apply(theta, y, h)
