"""Differentiable focal intensities: torch.autograd.Function over ofa_forward / ofa_adjoint.

FocusIntensity.apply(phi, plan) returns I_k = |Theta_k|^2 for the CGH phi
(device [ny][nx] float32), Theta = Eq. 2 at the plan's foci with the plan's
amplitude.  Its backward calls the library's adjoint kernel: given
g = dL/dI it returns dL/dphi = 2 Im(conj(E) B), B = P_MTP^H(g * Theta), the
same inverse product the GSW loop uses.  Any loss written in torch on the
intensities can then drive gradient-based CGH optimisation beside the GSW loop
(for example the intensity loss sum_k (I_k / sum I - t_k)^2).
"""
from __future__ import annotations

import torch

from . import ofa


class FocusIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi: torch.Tensor, plan: "ofa.Plan"):
        if not phi.is_cuda or phi.dtype != torch.float32:
            raise TypeError("phi must be a float32 CUDA tensor")
        phi = phi.contiguous()
        theta = torch.empty(plan.K, 2, dtype=torch.float32, device=phi.device)
        inten = torch.empty(plan.K, dtype=torch.float32, device=phi.device)
        ofa.ofa_forward(plan.handle, phi, theta, inten)
        ctx.save_for_backward(phi, theta)
        ctx.plan = plan
        return inten

    @staticmethod
    def backward(ctx, grad_inten: torch.Tensor):
        phi, theta = ctx.saved_tensors
        grad_phi = torch.empty_like(phi)
        ofa.ofa_adjoint(ctx.plan.handle, phi, theta, grad_inten.contiguous().float(), grad_phi)
        return grad_phi, None


def focus_intensity(phi: torch.Tensor, plan: "ofa.Plan") -> torch.Tensor:
    return FocusIntensity.apply(phi, plan)


def intensity_loss(inten: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """sum_k (I_k / sum I - t_k)^2 with t = target / sum target."""
    t = target / target.sum()
    return torch.sum((inten / inten.sum() - t) ** 2)


def optimize_adam(plan: "ofa.Plan", phi0: torch.Tensor, target: torch.Tensor, steps: int,
                  lr: float = 0.05, betas=(0.9, 0.999), eps: float = 1e-8):
    """Adam on phi for the intensity loss; returns (phi, per-step losses).

    The plan must have been created with stream=torch.cuda.current_stream().cuda_stream
    so that the library's kernels and torch's run in one order.
    """
    phi = phi0.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([phi], lr=lr, betas=betas, eps=eps)
    losses = torch.empty(steps, device=phi.device)
    for i in range(steps):
        opt.zero_grad(set_to_none=True)
        loss = intensity_loss(focus_intensity(phi, plan), target)
        loss.backward()
        opt.step()
        losses[i] = loss.detach()
    return phi.detach(), losses
