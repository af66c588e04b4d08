"""Objective J2 of Eq. objective2 (the oar, translating body: F_L + w_D F_D) on the CUDA path against the FP64 oracle.

The CUDA path uses the identity sum_j kappa^ref_j u^ref_j = sum_x kappa_n(x) u_n(x) (pinned in the oracle tests)
and injects the adjoint source g kappa_n before each adjoint step. Cases: both lattices, both precisions,
the checkpoint modes whose reverse sweeps run in segments, the fused two-step forward, and the gradient modes.
"""
import numpy as np
import pytest

from helpers import oracle_run, tiny_workload
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots
from test_gpu_parity import check

pytestmark = pytest.mark.gpu

OAR = dict(objective="J2", w_D=0.3, drag_span=9.0)
TOL = {"fp64": (1e-10, 1e-10, 1e-10), "fp32": (1e-4, 1e-4, 1e-3)}


# the oracle runs in FP64 whatever the path's precision, on inputs drawn from the seed and the shapes: one run per
# lattice serves both precisions (the J2 oracle forms dense weight matrices every step and takes minutes in 3D)
_ORACLE = {}


def oracle_for(w):
    if w["lattice"] not in _ORACLE:
        _ORACLE[w["lattice"]] = oracle_run(w, draw_gamma(w), draw_knots(w))
    return _ORACLE[w["lattice"]]


@pytest.mark.parametrize("lattice,prec", [("D2Q9", "fp64"), ("D3Q15", "fp64"), ("D2Q9", "fp32"), ("D3Q15", "fp32")])
def test_oar_objective_parity(lattice, prec):
    w = tiny_workload(lattice, precision=prec, **OAR)
    g, o = check(w, *TOL[prec], ref=oracle_for(w))
    assert abs(o["J"]) > 0 and np.abs(o["dknots"]).max() > 0


def test_oar_plane_pair_kernels_fp32():
    # J2 through the D3Q15 plane-pair kernels on a grid with a block inside it (the tile at x0 = 32, y0 = 8 fetches
    # by tensor copies): the recomputation's footprint factors, the sensitivity column kernel and design gather
    # (J2's kappa-bar term added after them).  Small, as the oracle's J2 forms dense weight matrices every step.
    w = tiny_workload("D3Q15", precision="fp32", tile_rows=128, tile_rows_adj=192, shape=(72, 20, 12),
                      design=(4, 4, 4), probe_lo=(50, 4, 3), probe_hi=(62, 16, 9), ckpt="sqrt", Nt=6, **OAR)
    g, o = check(w, *TOL["fp32"])
    assert g["stats"]["tile_rows_fwd"] == 128 and g["stats"]["tile_rows_adj"] == 192
    assert abs(o["J"]) > 0 and np.abs(o["dknots"]).max() > 0


@pytest.mark.parametrize("ckpt,rows", [("sqrt", 3), ("revolve", 1)])
def test_oar_checkpointed_reverse_sweeps(ckpt, rows):
    w = tiny_workload("D2Q9", precision="fp64", ckpt=ckpt, ckpt_slots=2, seg_len=4, tile_rows=rows, Nt=41, **OAR)
    g, _ = check(w, *TOL["fp64"])
    assert g["stats"]["recompute_steps"] > 0


@pytest.mark.parametrize("mode", ["shape", "motion"])
def test_oar_gradient_modes(mode):
    check(tiny_workload("D2Q9", precision="fp64", mode=mode, **OAR), *TOL["fp64"])
