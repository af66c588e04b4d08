"""Plain projected-gradient optimisation driver around the solver.

The paper optimises with MMA (Sec. 3), which is not part of this library.  This driver takes normalised ascent
steps on J (Eq. objective1 is maximised): gamma <- clip(gamma + s_g g / |g|_inf, 0, 1) and
knots <- clip(knots + s_p k / |k|_inf, -bound, bound), the 256x128x128 workload's "10 projected-gradient
iterations" (s_g = 0.05, s_p = 0.5 cell).  Every iteration is lks_forward_dev, lks_adjoint_dev and two
lks_gradient_step_dev calls on device arrays; J is read back once per iteration.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from .binding import LKSError, _stream_ptr


def gradient_step_dev(d_g, d_x, step: float, lo: float, hi: float, stream=None):
    """d_x <- clip(d_x + step * d_g / max|d_g|, lo, hi) in place (float64 CUDA tensors of equal size)."""
    lib = _abi.load()
    rc = lib.lks_gradient_step_dev(d_x.numel(), step, C.c_void_p(d_g.data_ptr()), C.c_void_p(d_x.data_ptr()),
                                   lo, hi, _stream_ptr(stream))
    if rc != 0:
        raise LKSError(rc, lib.lks_strerror(rc).decode())


def optimize(solver, gamma: np.ndarray, knots: np.ndarray, iters: int = 10, gamma_step: float = 0.05,
             pos_step: float = 0.5, pos_bound: float = np.inf, device=None):
    """Run `iters` ascent iterations from (gamma, knots); returns (gamma, knots, J of every iteration)."""
    import torch

    dev = device or torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    d_gamma = torch.tensor(np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).T), device=dev)
    d_knots = torch.tensor(np.asarray(knots, dtype=np.float64), device=dev)
    d_J = torch.empty((), dtype=torch.float64, device=dev)
    d_dg, d_dk = torch.empty_like(d_gamma), torch.empty_like(d_knots)
    history = []
    for _ in range(iters):
        solver.forward_dev(d_gamma, d_knots, d_J, stream=stream)
        solver.adjoint_dev(d_dg, d_dk, stream=stream)
        history.append(float(d_J.item()))
        gradient_step_dev(d_dg, d_gamma, gamma_step, 0.0, 1.0, stream=stream)
        gradient_step_dev(d_dk, d_knots, pos_step, -pos_bound, pos_bound, stream=stream)
    return d_gamma.cpu().numpy().T.copy(), d_knots.cpu().numpy(), history
