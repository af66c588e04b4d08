"""Parity where the method's claims live: full horizons, the periodic seam and a body crossing the wall planes.

- The 512x256 D2Q9 workload at its full 4000 steps: the FP32-state path against the plain FP64 GPU path on the
  same inputs (velocity <= 1e-4 max relative after the full horizon, gradients <= 1e-3 relative L2), and the FP32
  path against the FP64 oracle over 400 steps of the full grid.
- A body placed across the periodic seam x = 0 (the footprint box wraps; the transposed mapping folds design
  contributions across the seam): both lattices, both transfer kernels, both precisions, several step kernels.
- The 128x64x64 D3Q15 grid with the body displaced by the workload's full amplitude of 16 cells towards two walls,
  so that its footprint crosses the wall planes y = 63 and z = 0 (contributions outside the grid dropped, wall
  nodes imposed).
"""
import numpy as np
import pytest

from helpers import oracle_run, rel_l2, rel_max, tiny_workload
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots, workload
from test_gpu_parity import check, gpu_run

pytestmark = pytest.mark.gpu

FP64 = (1e-10, 1e-10, 1e-10)
FP32 = (1e-5, 1e-4, 1e-3)


def test_c2_full_horizon_fp32_against_fp64_gpu():
    # 4000 steps, sqrt(N) checkpoints, the launch configuration of the benchmark (autotuned variants)
    w32 = workload("d2q9_512x256_fp32")
    w64 = dict(w32, precision="fp64")
    gamma, knots = draw_gamma(w32), draw_knots(w32)
    a = gpu_run(w32, gamma, knots)
    b = gpu_run(w64, gamma, knots)
    assert abs(a["J"] - b["J"]) <= 1e-4 * abs(b["J"]), (a["J"], b["J"])
    assert rel_max(a["u"], b["u"]) <= 1e-4
    assert rel_max(a["p"], b["p"]) <= 1e-5
    assert rel_l2(a["dgamma"], b["dgamma"]) <= 1e-3
    assert rel_l2(a["dknots"], b["dknots"]) <= 1e-3
    assert abs(b["J"]) > 0 and np.linalg.norm(b["dgamma"]) > 0


def test_c2_full_grid_400_steps_fp32_against_oracle():
    # the full 512x256 grid over 400 steps (the motion amplitude scaled with the horizon, so body speeds match the
    # workload's; the probe box next to the body so that J and its gradients are not ~0)
    w = workload("d2q9_512x256_fp32", Nt=400, K=12, R_t=100.0, amp=32.0 * 400 / 4000, probe_lo=(300, 96),
                 probe_hi=(360, 160))
    check(w, *FP32)


SEAM2 = dict(base_center=(2.0, 18.0))
SEAM3 = dict(base_center=(1.5, 9.0, 6.0))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("rows", [1, 3, 8, 32])
def test_body_across_periodic_seam_d2q9(prec, kernel, rows):
    w = tiny_workload("D2Q9", precision=prec, kernel=kernel, tile_rows=rows, **SEAM2)
    g, o = check(w, *(FP64 if prec == "fp64" else FP32))
    # the design gradient has weight on both sides of the seam: the body really straddles x = 0
    assert np.abs(o["dgamma"]).max() > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("rows", [1, 8, 32])
def test_body_across_periodic_seam_d3q15(prec, kernel, rows):
    w = tiny_workload("D3Q15", precision=prec, kernel=kernel, tile_rows=rows, **SEAM3)
    check(w, *(FP64 if prec == "fp64" else FP32))


_C3_ORACLE = {}


@pytest.mark.parametrize("rows", [0, 8, 32])
def test_c3_body_crossing_wall_planes(rows):
    # the design centre 16 cells (the workload's amplitude) off the centre towards y = 63 and z = 0: the 52-node
    # extended design grid reaches y in [21.5, 73.5] and z in [-10.5, 41.5], across both wall planes
    w = workload("d3q15_128x64x64_fp32", Nt=12, K=4, R_t=3.0, amp=16.0 * 12 / 2000, seg_len=2,
                 base_center=(63.5, 47.5, 15.5), probe_lo=(100, 20, 20), probe_hi=(112, 44, 44))
    if "ref" not in _C3_ORACLE:  # the same inputs for every step-kernel variant
        _C3_ORACLE["ref"] = oracle_run(w, draw_gamma(w), draw_knots(w))
    g, o = check(dict(w, tile_rows=rows), *FP32, ref=_C3_ORACLE["ref"])
    assert np.abs(o["dgamma"]).max() > 0
