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


def lbm_loss(phi0: torch.Tensor, R: torch.Tensor, sim: LBM, T: int, target: torch.Tensor) -> torch.Tensor:
    """L = 1/2 sum_x (phi(x, T) - target(x))^2 with gradients through the adjoint kernels."""
    r = LBMFunction.apply(phi0, R, sim, T) - target
    return 0.5 * torch.dot(r, r)
