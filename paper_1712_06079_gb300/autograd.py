"""Differentiable rollout of the lattice Boltzmann step.

``rollout(lattice, rho0, Tr, G, nsteps)`` runs nsteps steps from f^eq(rho0, 0)
and returns the final density field; its backward pass is the hand-written
adjoint of the step in the CUDA library (``lbm_adjoint_forward`` /
``lbm_adjoint_backward``), with the forward states kept every
``checkpoint_interval`` steps (default ceil(sqrt(nsteps))) and recomputed in
between.  Gradients flow to rho0 and to the reduced temperature Tr; the
interaction strength G of the paper's Shan-Chen form cancels from Eq. 22, so
its gradient is zero.
"""
from __future__ import annotations

import math

import torch

from . import lbm


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, Tr, G, lattice, nsteps, checkpoint_interval):
        rho0 = rho0.contiguous()
        rhoT = torch.empty_like(rho0)
        torch.cuda.synchronize(rho0.device)
        lattice.adjoint_forward(rho0.data_ptr(), nsteps, checkpoint_interval, rhoT.data_ptr())
        lattice.sync()
        ctx.lattice = lattice
        ctx.tr_shape = Tr.shape
        ctx.g_shape = G.shape
        return rhoT

    @staticmethod
    def backward(ctx, grad_rhoT):
        g = grad_rhoT.contiguous()
        grad_rho0 = torch.empty_like(g)
        torch.cuda.synchronize(g.device)
        _, gTr = ctx.lattice.adjoint_backward(g.data_ptr(), grad_rho0.data_ptr())
        dtr = torch.full(ctx.tr_shape, gTr, dtype=torch.float64, device=g.device)
        dg = torch.zeros(ctx.g_shape, dtype=torch.float64, device=g.device)
        return grad_rho0, dtr, dg, None, None, None


def rollout(lattice: "lbm.Lattice", rho0: torch.Tensor, Tr: torch.Tensor, G: torch.Tensor, nsteps: int,
            checkpoint_interval: int | None = None) -> torch.Tensor:
    """Final density after nsteps steps, differentiable in rho0 and Tr.

    rho0: (ny, nx) CUDA tensor of the lattice precision.  Tr and G: scalar
    float64 tensors; Tr must equal the lattice's reduced temperature (the
    library context is built for one temperature)."""
    if not rho0.is_cuda:
        raise ValueError("rho0 must be a CUDA tensor")
    if abs(float(Tr.detach()) - lattice.params.Tr) > 1e-15 * max(1.0, abs(lattice.params.Tr)):
        raise ValueError("Tr must equal the lattice's reduced temperature")
    want = torch.float64 if lattice.params.prec == "f64" else torch.float32
    if rho0.dtype != want or tuple(rho0.shape) != lattice.shape:
        raise ValueError(f"rho0 must be a {tuple(lattice.shape)} {want} tensor")
    if checkpoint_interval is None:
        checkpoint_interval = max(1, math.ceil(math.sqrt(nsteps)))
    return _Rollout.apply(rho0, Tr, G, lattice, int(nsteps), int(checkpoint_interval))
