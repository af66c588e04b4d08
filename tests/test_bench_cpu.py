"""Host logic of bench.py (no GPU): the step-kernel name and sources a tile_rows code selects, and the committed ncu
traffic lines that the roofline's `traffic` field reads, which must belong to the kernels' current sources (a
kernel changed since its capture reports null traffic, so a stale line shows here first)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("lattice,rows,kind,name", [
    ("D3Q15", 128, "fwd", "fwd3p_kernel<ZB=16>"),
    ("D3Q15", 160, "fwd", "fwd3p_kernel<ZB=32>"),
    ("D3Q15", 192, "adj", "adj3p_kernel<ZB=64>"),
    ("D3Q15", 32, "fwd", "fwd3s_kernel<ZB=16,TY=8>"),
    ("D3Q15", 1, "adj", "adj_step_kernel"),
    ("D2Q9", 32, "fwd", "fwd2v_kernel<R=32>"),
    ("D2Q9", 64, "adj", "adj2v_kernel<R=64>"),
    ("D2Q9", 3, "fwd", "fwd2r2_kernel"),
    ("D2Q9", 8, "adj", "adj2d_kernel<R=8>"),
])
def test_kernel_variant_names(lattice, rows, kind, name):
    got, src, per_launch = bench.kernel_variant(lattice, rows, kind)
    assert got == name
    files = src if isinstance(src, (list, tuple)) else [src]
    for f in files:
        assert os.path.exists(os.path.join(ROOT, "paper_2608_01071_b300", "csrc", f)), f
    assert per_launch == (2 if (lattice, rows) == ("D2Q9", 3) else 1)


def test_plane_pair_sources_cover_their_headers():
    # the plane-pair kernels use the tensor-copy and separable headers: a change there must invalidate the capture
    _, src, _ = bench.kernel_variant("D3Q15", 128, "fwd")
    assert {"lks_tma.cuh", "lks_step3s.cuh", "lks_step3p.cuh"} <= set(src)


@pytest.mark.parametrize("workload,lattice,rows,kind", [
    ("d3q15_256x128x128_fp32", "D3Q15", 128, "fwd"),
    ("d3q15_256x128x128_fp32", "D3Q15", 160, "fwd"),
    ("d3q15_256x128x128_fp32", "D3Q15", 192, "adj"),
    ("d2q9_4096x4096_fp32", "D2Q9", 32, "fwd"),
    ("d2q9_4096x4096_fp32", "D2Q9", 64, "adj"),
])
def test_committed_traffic_matches_current_sources(workload, lattice, rows, kind):
    name, src, _ = bench.kernel_variant(lattice, rows, kind)
    t = bench.captured_traffic(workload, name, src)
    assert t is not None, f"no ncu traffic line for {name} of the current sources in profiles/step_kernels_{workload}.md"
    assert 50e6 < t < 1e9
