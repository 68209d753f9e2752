"""torch.autograd.Function around the forward model and its hand-written adjoint.

    p = proj_warp(ctx, model_id, w, angle)      # p = P f(mean + U w)   [nv][nu]
    loss(p).backward()                          # w.grad = (dp/dw)^T dloss/dp

forward calls pr_forward (fused DVF synthesis + warp, then the ray-march
projector); backward calls pr_vjp, which warps to get h_k = (df/dx) . u_k and
runs the gather transpose P^T contracted with h_k, never storing P^T grad_p
(the gradient formula after Eq. 4 without the factor 2 of J).
"""

from __future__ import annotations

import numpy as np
import torch


class ProjWarp(torch.autograd.Function):
    @staticmethod
    def forward(fctx, w, context, model_id: int, angle: float):
        w_host = w.detach().to("cpu", torch.float64).numpy()
        p = context.forward(model_id, w_host, angle)
        fctx.context, fctx.model_id, fctx.angle = context, model_id, angle
        fctx.w_host = w_host
        fctx.w_meta = (w.dtype, w.device)
        return p

    @staticmethod
    def backward(fctx, grad_p):
        g = fctx.context.vjp(fctx.model_id, fctx.w_host, fctx.angle, grad_p.detach().float().contiguous())
        dtype, device = fctx.w_meta
        return torch.as_tensor(np.asarray(g), dtype=dtype, device=device), None, None, None


def proj_warp(context, model_id: int, w: torch.Tensor, angle: float) -> torch.Tensor:
    """Differentiable projection of the model warped at PCA coefficients w (K,)."""
    if w.dim() != 1 or w.numel() != context.K(model_id):
        raise ValueError("w must be a vector of the model's K coefficients")
    return ProjWarp.apply(w, context, model_id, float(angle))
