"""torch.autograd.Function over the refinement loss kernels.

Forward: L_roi(omega) = sum_v (S[roi, v] - I(alpha, beta of R^T u_v))^2 with
R = exp([omega]x) R(q0), evaluated by the library's forward kernel; backward:
dL/domega from the library's hand-written backward kernel (bilinear image
gradient, chain rule through the elevation-azimuth angles and the SO(3) left
Jacobian).  Marshalling only: both passes run in CUDA kernels.
"""
from __future__ import annotations

import torch

from . import aptidx_refine_loss


class RefineLoss(torch.autograd.Function):
    """loss[roi] (float32) of axis-angle offsets omega [nroi, 3] (float64,
    CUDA) from reference orientations q0 [nroi, 4] (float64, CUDA), for
    measured signatures S [nroi, nv] (float32, CUDA) against candidate
    `cand` of context `handle`."""

    @staticmethod
    def forward(fctx, omega, S, q0, handle, cand):
        omega = omega.detach().contiguous()
        loss = torch.empty(omega.shape[0], dtype=torch.float32, device=omega.device)
        aptidx_refine_loss(handle, cand, S, q0, loss, None, omega)
        fctx.save_for_backward(omega, S, q0)
        fctx.handle = handle
        fctx.cand = cand
        return loss

    @staticmethod
    def backward(fctx, grad_loss):
        omega, S, q0 = fctx.saved_tensors
        loss = torch.empty(omega.shape[0], dtype=torch.float32, device=omega.device)
        grad = torch.empty((omega.shape[0], 3), dtype=torch.float32, device=omega.device)
        aptidx_refine_loss(fctx.handle, fctx.cand, S, q0, loss, grad, omega)
        g = grad.to(torch.float64) * grad_loss.to(torch.float64)[:, None]
        return g, None, None, None, None


def refine_loss(omega, S, q0, handle, cand: int = 0):
    return RefineLoss.apply(omega, S, q0, handle, cand)
