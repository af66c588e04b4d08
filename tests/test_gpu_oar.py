"""Objective J2 of Eq. objective2 (the oar, translating body: F_L + w_D F_D) on the CUDA path against the FP64 oracle.

The CUDA path uses the identity sum_j kappa^ref_j u^ref_j = sum_x kappa_n(x) u_n(x) (pinned in the oracle tests)
and injects the adjoint source g kappa_n before each adjoint step. Cases: both lattices, both precisions,
the checkpoint modes whose reverse sweeps run in segments, the fused two-step forward, and the gradient modes.
"""
import numpy as np
import pytest

from helpers import tiny_workload
from test_gpu_parity import check

pytestmark = pytest.mark.gpu

OAR = dict(objective="J2", w_D=0.3, drag_span=9.0)
TOL = {"fp64": (1e-10, 1e-10, 1e-10), "fp32": (1e-4, 1e-4, 1e-3)}


@pytest.mark.parametrize("lattice,prec", [("D2Q9", "fp64"), ("D3Q15", "fp64"), ("D2Q9", "fp32")])
def test_oar_objective_parity(lattice, prec):
    g, o = check(tiny_workload(lattice, precision=prec, **OAR), *TOL[prec])
    assert abs(o["J"]) > 0 and np.abs(o["dknots"]).max() > 0


@pytest.mark.parametrize("ckpt,rows", [("sqrt", 3), ("revolve", 1)])
def test_oar_checkpointed_reverse_sweeps(ckpt, rows):
    w = tiny_workload("D2Q9", precision="fp64", ckpt=ckpt, ckpt_slots=2, seg_len=4, tile_rows=rows, Nt=41, **OAR)
    g, _ = check(w, *TOL["fp64"])
    assert g["stats"]["recompute_steps"] > 0


@pytest.mark.parametrize("mode", ["shape", "motion"])
def test_oar_gradient_modes(mode):
    check(tiny_workload("D2Q9", precision="fp64", mode=mode, **OAR), *TOL["fp64"])
