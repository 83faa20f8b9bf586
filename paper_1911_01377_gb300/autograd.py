"""The u-series energy as a differentiable PyTorch function.

    E = usr_energy(xyz, q, ctx)          # xyz (n, 3), q (n,) float32 CUDA tensors
    E.backward()                         # xyz.grad = dE/dx = -F, q.grad = dE/dq = phi

The forward pass is one `usr_eval` (all of it in libusr's kernels); the
backward pass launches nothing on the device beyond the scaling of the saved
outputs: the evaluation already produced F_i = -dE/dr_i and phi_i = dE/dq_i.
phi is the derivative of E as a quadratic form of the charges, which holds off
the neutral manifold too because the k = 0 term is dropped (Eq. 4 sums k != 0).
Second derivatives are not provided.
"""
from __future__ import annotations

import torch

from .usr import USeries


class UsrEnergy(torch.autograd.Function):
    """Energy (float64 scalar) of positions `xyz` and charges `q` with a hand-written backward."""

    @staticmethod
    def forward(fctx, xyz: torch.Tensor, q: torch.Tensor, ctx: USeries):
        if not (xyz.is_cuda and q.is_cuda and xyz.dtype == torch.float32 and q.dtype == torch.float32):
            raise TypeError("usr_energy: xyz and q must be float32 CUDA tensors")
        if xyz.dim() != 2 or xyz.shape[1] != 3 or q.shape != (xyz.shape[0],):
            raise ValueError("usr_energy: xyz must be (n, 3) and q (n,)")
        xyzq = torch.cat([xyz.detach(), q.detach()[:, None]], dim=1).contiguous()
        out, en = ctx.eval(xyzq)
        fctx.save_for_backward(out)
        fctx.mark_non_differentiable(en)
        return en[0].clone(), en

    @staticmethod
    def backward(fctx, g_energy, g_parts):
        (out,) = fctx.saved_tensors
        g = g_energy.to(torch.float32)
        gx = -g * out[:, :3] if fctx.needs_input_grad[0] else None
        gq = g * out[:, 3] if fctx.needs_input_grad[1] else None
        return gx, gq, None


def usr_energy(xyz: torch.Tensor, q: torch.Tensor, ctx: USeries, parts: bool = False):
    """E(xyz, q) as a differentiable float64 scalar; with parts=True also the
    (E, E_near, E_far, E_self) breakdown (not differentiable)."""
    e, en = UsrEnergy.apply(xyz, q, ctx)
    return (e, en) if parts else e
