"""torch.autograd.Function over the batched log-likelihood: the forward pass runs the library's
gradient kernels (log L and d logL/d theta in one call) and keeps the gradient; the backward pass
scales it by the incoming cotangent. Differentiation follows Sec. 2.3 of arXiv:2602.12011
(gradients of the likelihood for gradient-based sampling), with a hand-written adjoint in place
of the paper's automatic differentiation."""
from __future__ import annotations

import torch

from . import _lib


class LogLikelihood(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, dets, mode_mask: int):
        if not theta.is_cuda or theta.dtype != torch.float64:
            raise TypeError("theta must be a float64 CUDA tensor [B][11]")
        res = _lib.loglike_grad(dets, theta.detach(), mode_mask)
        ctx.save_for_backward(res["grad"])
        return res["logl"]

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return g.reshape(-1, 1) * grad, None, None


def loglike(theta: torch.Tensor, dets, mode_mask: int) -> torch.Tensor:
    """log L(theta) [B], differentiable with respect to theta [B][11]."""
    return LogLikelihood.apply(theta, dets, mode_mask)
