"""Differentiable focal intensities and gradient-based CGH optimisation.

The loop AdamLoop runs by default is library kernels only (ofa_forward,
ofa_loss_adjoint, ofa_adam_step); FocusIntensity exposes the same products to torch
autograd for other losses.

Differentiable focal intensities: torch.autograd.Function over ofa_forward / ofa_adjoint.

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


def _same_stream(plan) -> bool:
    return getattr(plan, "stream", None) == torch.cuda.current_stream().cuda_stream


class FocusIntensity(torch.autograd.Function):
    """The library runs on the plan's stream; when that is not torch's current stream the
    calls synchronise the device around the library work (correct, but slower than
    creating the plan on the stream the torch work runs on)."""

    @staticmethod
    def forward(ctx, phi: torch.Tensor, plan: "ofa.Plan"):
        if not phi.is_cuda or phi.dtype != torch.float32:
            raise TypeError("phi must be a float32 CUDA tensor")
        phi = phi.contiguous()
        theta = torch.empty(plan.K, 2, dtype=torch.float32, device=phi.device)
        inten = torch.empty(plan.K, dtype=torch.float32, device=phi.device)
        same = _same_stream(plan)
        if not same:
            torch.cuda.synchronize()
        ofa.ofa_forward(plan.handle, phi, theta, inten)
        if not same:
            torch.cuda.synchronize()
        ctx.save_for_backward(phi, theta)
        ctx.plan = plan
        return inten

    @staticmethod
    def backward(ctx, grad_inten: torch.Tensor):
        phi, theta = ctx.saved_tensors
        grad_phi = torch.empty_like(phi)
        g = grad_inten.contiguous().float()
        same = _same_stream(ctx.plan)
        if not same:
            torch.cuda.synchronize()
        ofa.ofa_adjoint(ctx.plan.handle, phi, theta, g, grad_phi)
        if not same:
            torch.cuda.synchronize()
        return grad_phi, None


def focus_intensity(phi: torch.Tensor, plan: "ofa.Plan") -> torch.Tensor:
    return FocusIntensity.apply(phi, plan)


def intensity_loss(inten: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """sum_k (I_k / sum I - t_k)^2 with t = target / sum target."""
    t = target / target.sum()
    return torch.sum((inten / inten.sum() - t) ** 2)


class AdamLoop:
    """Adam on phi for the intensity loss, one step at a time or as a CUDA graph.

    library=True (default): every step is library kernels only -- ofa_forward (field
    planes, forward product, focal output), ofa_loss_adjoint (loss, dL/dI, inverse
    product with the gradient epilogue) and ofa_adam_step (update, step counter), with
    the loss of each step written by the library into `losses`.  library=False runs the
    loss and Adam in torch through FocusIntensity (autograd over the same products).

    The plan must enqueue on the stream the torch work runs on: `stream` if given
    (the plan created with stream=stream.cuda_stream), else torch's current stream.
    graph=True captures one whole step in a CUDA graph that run() replays; one eager
    step first creates the optimiser state and the plan's field planes and is then
    undone, so the trajectory is the eager one.  A graph needs a stream other than
    the legacy default stream.
    """

    def __init__(self, plan: "ofa.Plan", phi0: torch.Tensor, target: torch.Tensor,
                 max_steps: int, lr: float = 0.05, betas=(0.9, 0.999), eps: float = 1e-8,
                 stream: torch.cuda.Stream | None = None, graph: bool = False,
                 library: bool = True):
        self.plan, self.target = plan, target
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.graph = None
        self.library = library
        self.lr, self.betas, self.eps = float(lr), betas, float(eps)
        if library:
            self._init_library(phi0, max_steps, graph)
            return
        with torch.cuda.stream(self.stream):
            self.phi = phi0.detach().clone().requires_grad_(True)
            self.losses = torch.zeros(max_steps, device=self.phi.device)
            self.idx = torch.zeros(1, dtype=torch.long, device=self.phi.device)
            self.opt = torch.optim.Adam([self.phi], lr=lr, betas=betas, eps=eps,
                                        capturable=graph)
            if graph:
                self._step()           # warm-up: optimiser state, field planes
                with torch.no_grad():
                    self.phi.copy_(phi0)
                    for st in self.opt.state.values():
                        for v in st.values():
                            v.zero_()
                    self.idx.zero_()
                self.opt.zero_grad(set_to_none=True)
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph, stream=self.stream):
                    self._step()

    def _init_library(self, phi0, max_steps, graph):
        dev = phi0.device
        if graph and getattr(self.plan, "stream", None) != self.stream.cuda_stream:
            raise ValueError("graph=True needs the plan created on the loop's stream "
                             "(Plan(..., stream=stream.cuda_stream))")
        with torch.cuda.stream(self.stream):
            self.phi = phi0.detach().clone().contiguous()
            self.m = torch.zeros_like(self.phi)
            self.v = torch.zeros_like(self.phi)
            self.step = torch.zeros(1, dtype=torch.int32, device=dev)
            self.theta = torch.empty(self.plan.K, 2, dtype=torch.float32, device=dev)
            self.inten = torch.empty(self.plan.K, dtype=torch.float32, device=dev)
            self.grad = torch.empty_like(self.phi)
            self.losses = torch.zeros(max_steps + 1, device=dev)
            # the library runs on the plan's stream: these buffers must be ready for it
            torch.cuda.synchronize()
            if graph:
                self._step_library()       # warm-up: the plan's field planes
                self.phi.copy_(phi0)
                self.m.zero_()
                self.v.zero_()
                self.step.zero_()
                self.losses.zero_()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph, stream=self.stream):
                    self._step_library()

    def _step_library(self):
        h = self.plan.handle
        ofa.ofa_forward(h, self.phi, self.theta, self.inten)
        ofa.ofa_loss_adjoint(h, self.phi, self.theta, self.grad, self.losses, self.step)
        ofa.ofa_adam_step(h, self.phi, self.grad, self.m, self.v, self.step, self.lr,
                          self.betas[0], self.betas[1], self.eps)

    def _step(self):
        loss = intensity_loss(focus_intensity(self.phi, self.plan), self.target)
        loss.backward()
        self.opt.step()
        self.losses.index_copy_(0, self.idx, loss.detach().view(1))
        self.idx.add_(1)

    def run(self, steps: int):
        """Enqueue `steps` Adam steps (no synchronisation)."""
        with torch.cuda.stream(self.stream):
            for _ in range(steps):
                if self.graph is not None:
                    self.graph.replay()
                elif self.library:
                    self._step_library()
                else:
                    self.opt.zero_grad(set_to_none=True)
                    self._step()


def optimize_adam(plan: "ofa.Plan", phi0: torch.Tensor, target: torch.Tensor, steps: int,
                  lr: float = 0.05, betas=(0.9, 0.999), eps: float = 1e-8,
                  stream: torch.cuda.Stream | None = None, graph: bool = False,
                  library: bool = True):
    """`steps` Adam steps from phi0; returns (phi, the loss before each step) (see
    AdamLoop)."""
    loop = AdamLoop(plan, phi0, target, steps, lr, betas, eps, stream, graph, library)
    loop.run(steps)
    if getattr(plan, "stream", None) != loop.stream.cuda_stream:
        torch.cuda.synchronize()       # the library worked on the plan's own stream
    return loop.phi.detach(), loop.losses[:steps]
