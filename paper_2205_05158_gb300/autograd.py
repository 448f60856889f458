"""torch.autograd.Function over the library's forward chain and hand-written adjoint.

fddpd_loss(theta, plan, s, H, W, alpha, pa) returns the training criterion of Sec. V-A
(mean |y/alpha - s|^2 over the data subcarriers of every symbol) as a 0-dim CUDA tensor
whose gradient with respect to theta is computed by fddpd_backward: the library re-runs
the forward chain and applies the adjoint of the combine, DFT, PA, IDFT, precoder and
FD-CNN stages; no activation or time-domain signal is kept between the two passes.
Only theta is differentiable; the symbols, channel, precoder and PA are data.
"""
from __future__ import annotations

import torch


class FddpdLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, plan, s, H, W, alpha, pa):
        th = theta.detach().contiguous()
        met = torch.zeros(5, dtype=torch.float64, device=theta.device)
        plan.distort(s, H, W, alpha, pa, th, None, met)
        ctx.plan = plan
        ctx.save_for_backward(th, s, H, W, alpha, pa)
        return met[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        th, s, H, W, alpha, pa = ctx.saved_tensors
        g = torch.empty_like(th)
        ctx.plan.backward(s, H, W, alpha, pa, th, g)
        return grad_out * g, None, None, None, None, None, None


def fddpd_loss(theta, plan, s, H, W, alpha, pa):
    """Differentiable loss of the FD-DPD chain with respect to theta."""
    return FddpdLoss.apply(theta, plan, s, H, W, alpha, pa)
