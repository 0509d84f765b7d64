"""Differentiable rollout of the lattice Boltzmann step.

``rollout(lattice, rho0, Tr, G, nsteps)`` runs nsteps steps from f^eq(rho0, 0)
and returns the final density field; its backward pass is the hand-written
adjoint of the step in the CUDA library (``lbm_adjoint_forward`` /
``lbm_adjoint_backward``), with the forward states kept every
``checkpoint_interval`` steps (default ceil(sqrt(nsteps))) and recomputed in
between.  Gradients flow to rho0 and to the model's scalar parameter: with an
equation of state to the reduced temperature Tr (the interaction strength G
cancels from Eq. 22, so its gradient is zero); with the original effective
mass of Eq. 4 (eos "psi_exp") to G (there is no temperature).
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
        _, gTr, gG = ctx.lattice.adjoint_backward(g.data_ptr(), grad_rho0.data_ptr())
        dtr = torch.full(ctx.tr_shape, gTr, dtype=torch.float64, device=g.device)
        dg = torch.full(ctx.g_shape, gG, dtype=torch.float64, device=g.device)
        return grad_rho0, dtr, dg, None, None, None


def rollout(lattice: "lbm.Lattice", rho0: torch.Tensor, Tr: torch.Tensor, G: torch.Tensor, nsteps: int,
            checkpoint_interval: int | None = None) -> torch.Tensor:
    """Final density after nsteps steps, differentiable in rho0 and Tr.

    rho0: (ny, nx) CUDA tensor of the lattice precision.  Tr and G: scalar
    float64 tensors equal to the lattice's reduced temperature and (eos
    "psi_exp") interaction strength: the library context is built for one
    parameter set."""
    if not rho0.is_cuda:
        raise ValueError("rho0 must be a CUDA tensor")
    psi = lattice.params.eos == "psi_exp"
    if not psi and abs(float(Tr.detach()) - lattice.params.Tr) > 1e-15 * max(1.0, abs(lattice.params.Tr)):
        raise ValueError("Tr must equal the lattice's reduced temperature")
    if psi and abs(float(G.detach()) - lattice.params.G) > 1e-15 * max(1.0, abs(lattice.params.G)):
        raise ValueError("G must equal the lattice's interaction strength")
    want = torch.float64 if lattice.params.prec == "f64" else torch.float32
    if rho0.dtype != want or tuple(rho0.shape) != lattice.shape:
        raise ValueError(f"rho0 must be a {tuple(lattice.shape)} {want} tensor")
    if checkpoint_interval is None:
        checkpoint_interval = max(1, math.ceil(math.sqrt(nsteps)))
    return _Rollout.apply(rho0, Tr, G, lattice, int(nsteps), int(checkpoint_interval))
