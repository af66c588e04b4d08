"""torch.autograd.Function over the library's device entry points: forward = lks_forward_dev (returns J),
backward = lks_adjoint_dev (the hand-written discrete-adjoint kernels), on the current CUDA stream."""
from __future__ import annotations

import torch

from .binding import Solver


def _to_flat(t: torch.Tensor) -> torch.Tensor:
    # math order [x, y(, z)] -> library order (x fastest)
    return t.permute(*reversed(range(t.dim()))).contiguous()


def _from_flat(t: torch.Tensor) -> torch.Tensor:
    return t.permute(*reversed(range(t.dim())))


class LKSFunction(torch.autograd.Function):
    """J = LKSFunction.apply(gamma, knots, solver); gamma (design grid, float64, CUDA), knots (K, d) float64."""

    @staticmethod
    def forward(ctx, gamma, knots, solver: Solver):
        stream = torch.cuda.current_stream(gamma.device)
        J = torch.empty((), dtype=torch.float64, device=gamma.device)
        solver.forward_dev(_to_flat(gamma.detach()), knots.detach().contiguous(), J, stream=stream)
        ctx.solver = solver
        ctx.shape = gamma.shape
        return J

    @staticmethod
    def backward(ctx, grad_J):
        s = ctx.solver
        dev = grad_J.device
        stream = torch.cuda.current_stream(dev)
        dg = torch.empty(tuple(reversed(ctx.shape)), dtype=torch.float64, device=dev)
        dk = torch.empty((s.K, s.d), dtype=torch.float64, device=dev)
        s.adjoint_dev(dg, dk, stream=stream)
        return grad_J * _from_flat(dg), grad_J * dk, None
