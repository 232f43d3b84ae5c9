"""torch.autograd bindings of the library's discrete adjoint.

The lattice Boltzmann step is affine in the populations: f*(n+1) = C S f*(n) + dt omega R with a
per-site collision C and the streaming permutation S, so the transpose of T steps does not depend
on the forward states. The backward pass therefore runs T adjoint steps straight from the cotangent
of the outputs, with no stored trajectory and no forward recomputation; the forward pass keeps
nothing but the handle.
"""
from __future__ import annotations

import torch

from . import LBM


class LBMFunction(torch.autograd.Function):
    """phi(T) = F(phi0, R) for a periodic LBM handle; gradients w.r.t. phi0 and the source field R(x).

    The initial populations use the handle's init order with the finite-difference gradient of
    phi0, whose transpose is part of dL/dphi0."""

    @staticmethod
    def forward(ctx, phi0: torch.Tensor, R: torch.Tensor, sim: LBM, T: int):
        sim.init(phi0.detach().contiguous(), None, R.detach().contiguous())
        sim.step(T)
        ctx.sim, ctx.T = sim, int(T)
        return sim.macro()

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        sim = ctx.sim
        sim.adjoint_seed(g.contiguous())
        sim.adjoint_step(ctx.T)
        gphi0, _, gR = sim.adjoint_grads(want_grad=False, want_R=bool(ctx.needs_input_grad[1]))
        return gphi0, gR, None, None


class LBMBoxFunction(torch.autograd.Function):
    """phi(T) = F(phi0, grad phi0, jets) for a Dirichlet box (either precision) whose boundary data are given
    as jets, one (P, jet_len(d)) block per step at sim.boundary_points() (jets: (T, P, jet_len(d))).
    Gradients w.r.t. all three: the adjoint steps run from the cotangent of phi(T), the cotangent of
    each step's jets is read before its adjoint step (Eq. (bun1) / Eq. (bun2) transposed), and the
    transpose of the initialisation gives those of phi0 and grad phi0."""

    @staticmethod
    def forward(ctx, phi0: torch.Tensor, grad: torch.Tensor, jets: torch.Tensor, sim: LBM):
        jets = jets.detach().contiguous()
        sim.init(phi0.detach().contiguous(), grad.detach().contiguous())
        for n in range(jets.shape[0]):
            sim.set_boundary_jet(jets[n])
            sim.step(1)
        ctx.sim, ctx.shape = sim, tuple(jets.shape)
        ctx.shapes = (phi0.shape, grad.shape)
        return sim.macro()

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        sim = ctx.sim
        sim.adjoint_seed(g.contiguous())
        gjets = torch.empty(ctx.shape, dtype=torch.float64, device=g.device)
        for n in range(ctx.shape[0] - 1, -1, -1):
            sim.adjoint_jet_grad(out=gjets[n])
            sim.adjoint_step(1)
        gphi0, ggrad, _ = sim.adjoint_grads(want_grad=True, want_R=False)
        return gphi0.view(ctx.shapes[0]), ggrad.view(ctx.shapes[1]), gjets, None


def lbm_loss(phi0: torch.Tensor, R: torch.Tensor, sim: LBM, T: int, target: torch.Tensor) -> torch.Tensor:
    """L = 1/2 sum_x (phi(x, T) - target(x))^2 with gradients through the adjoint kernels."""
    r = LBMFunction.apply(phi0, R, sim, T) - target
    return 0.5 * torch.dot(r, r)
