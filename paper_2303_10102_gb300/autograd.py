"""The approximate negative log-likelihood as a differentiable PyTorch function.

The paper states that the HODLR construction can be differentiated (Sec. 3.3) and computes
the score from the derivative matrices K~_j of Alg. 2 with exact traces (Sec. 4.3,
App. B).  ``hodlr_nll`` exposes that computation to autograd:

* forward: L(theta) = N/2 log 2 pi + 1/2 log det K~ + 1/2 y^T K~^{-1} y (eq. log-like
  approximated), one build and factorization through the C ABI;
* backward with respect to theta: the score dL/dtheta_j = 1/2 tr(K~^{-1} K~_j)
  - 1/2 alpha^T K~_j alpha (eq. score approximated), computed in the same call as the
  forward value by the library (tangent sweeps of Alg. 2 for ell and kappa, closed forms
  for sigma^2 and tau^2);
* backward with respect to y: dL/dy = K~^{-1} y, one more solve with the stored factors.

With four parameters the tangent (forward-mode) sweeps cost less than a reverse sweep would,
and they are the exact derivative of the same K~(theta), so the autograd gradient is the
library's gradient.  Nothing here computes on the host: every value comes from the CUDA
library.
"""
from __future__ import annotations

import numpy as np
import torch


class _HodlrNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, y, h):
        th = theta.detach().to("cpu", torch.float64).numpy()
        nll, grad = h.nll_grad(th, y.detach())
        ctx.h, ctx.th = h, th
        ctx.save_for_backward(y)
        ctx.grad_theta = torch.as_tensor(np.asarray(grad, dtype=np.float64))
        return torch.tensor(nll, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (y,) = ctx.saved_tensors
        g_theta = g_y = None
        if ctx.needs_input_grad[0]:
            g_theta = (gout.to(torch.float64) * ctx.grad_theta)
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
