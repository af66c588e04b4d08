"""The objective J1 = E - phi V of Eq. objective1 with the variance term on (phi != 0), CUDA path vs the FP64 oracle.

The probe boxes reach a wall plane (wall nodes are not part of O_target) and the direction n has two non-zero
components, so that every term of the per-node source 1 + 2 phi E - 2 phi n.u is exercised.  phi is chosen so that
2 phi std(n.u) is about one: the variance then changes the gradient by O(1).  Tolerances as in the parity tests.
"""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_problem, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots
from test_gpu_parity import check, gpu_run

pytestmark = pytest.mark.gpu

VAR = {"D2Q9": dict(probe_lo=(50, 0), probe_hi=(62, 27), direction=(0.6, -0.8), phi_var=150.0),
       "D3Q15": dict(probe_lo=(30, 4, 0), probe_hi=(36, 14, 10), direction=(0.0, 0.6, 0.8), phi_var=1000.0)}
TOL = {"fp64": (1e-10, 1e-10, 1e-10), "fp32": (1e-5, 1e-4, 1e-3)}


def var_workload(lattice, **over):
    return tiny_workload(lattice, **dict(VAR[lattice], **over))


def oracle_terms(w, gamma, knots):
    P = oracle_problem(w)
    J, states = O.solve(P, gamma, knots, store=True)
    wO = O.probe_mean_weights(P)
    E = sum((wO * O.flow_along(P, u)).sum() for _, u in states[1:])
    S2 = sum((wO * O.flow_along(P, u) ** 2).sum() for _, u in states[1:])
    return J, E, S2 - E * E


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_variance_objective_parity(lattice, prec):
    w = var_workload(lattice, precision=prec)
    check(w, *TOL[prec])
    # E and V themselves, and J = E - phi V
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    J = s.forward(gamma, knots)
    E, V = s.objective_terms()
    s.close()
    Jo, Eo, Vo = oracle_terms(w, gamma, knots)
    tol = TOL[prec][0]
    assert abs(E - Eo) <= tol * abs(Eo) and abs(V - Vo) <= 10 * tol * abs(Vo), (E, Eo, V, Vo)
    assert abs(J - (E - w["phi_var"] * V)) <= 1e-14 * (abs(E) + w["phi_var"] * abs(V))
    assert abs(w["phi_var"] * Vo) > 0.3 * abs(Eo)  # the variance term is not negligible


@pytest.mark.parametrize("rows,prec", [(1, "fp64"), (2, "fp64"), (3, "fp64"), (4, "fp64"), (8, "fp64"), (32, "fp64"),
                                       (16, "fp32"), (64, "fp32")])
def test_variance_d2q9_kernel_variants(rows, prec):
    # the objective partials and the source in every D2Q9 step-kernel family (odd horizon: the two-step kernels
    # end on a single step)
    w = var_workload("D2Q9", precision=prec, tile_rows=rows, shape=(94, 45), probe_lo=(60, 0), probe_hi=(75, 30),
                     ckpt="sqrt", Nt=41)
    g, _ = check(w, *TOL[prec])
    assert g["stats"]["tile_rows_fwd"] == rows and g["stats"]["tile_rows_adj"] == rows


@pytest.mark.parametrize("rows", [1, 8, 16, 32, 64, 96])
def test_variance_d3q15_kernel_variants(rows):
    w = var_workload("D3Q15", tile_rows=rows, shape=(41, 21, 19), probe_lo=(28, 3, 0), probe_hi=(37, 15, 12),
                     ckpt="sqrt", Nt=24)
    g, _ = check(w, *TOL["fp64"])
    assert g["stats"]["tile_rows_fwd"] == rows


@pytest.mark.parametrize("fwd,adj", [(128, 128), (160, 192)])
def test_variance_d3q15_plane_pair_fp32(fwd, adj):
    # the objective partials and the variance source in the plane-pair kernels (FP32 only), on a grid with a
    # tensor-copy tile (x0 = 32, y0 = 8)
    w = var_workload("D3Q15", precision="fp32", tile_rows=fwd, tile_rows_adj=adj, shape=(72, 20, 24),
                     probe_lo=(40, 4, 6), probe_hi=(50, 16, 18), ckpt="sqrt", Nt=16)
    g, _ = check(w, *TOL["fp32"])
    assert g["stats"]["tile_rows_fwd"] == fwd and g["stats"]["tile_rows_adj"] == adj


@pytest.mark.parametrize("ckpt", ["revolve", "sqrt"])
def test_variance_graph_replay_new_inputs(ckpt):
    # the source constant 1 + 2 phi E is read on the device by the captured adjoint: replays with other inputs
    # (another E) must match fresh eager runs bit for bit
    w = var_workload("D2Q9", precision="fp32", ckpt=ckpt, ckpt_slots=2, seg_len=4, tile_rows=1)
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    s.set_graphs(True)
    for g_, k_ in [(gamma, knots), (gamma * 0.5, knots + 0.3), (gamma, knots)]:
        J = s.forward(g_, k_)
        dg, dk = s.adjoint()
        e = gpu_run(w, g_, k_)
        assert J == e["J"] and np.array_equal(dg, e["dgamma"]) and np.array_equal(dk, e["dknots"])
    s.close()


@pytest.mark.parametrize("rows", [1, 3])
def test_phi_zero_is_the_mean(rows):
    # phi = 0 gives J = E exactly; the squares are not summed and V is NaN
    w = var_workload("D2Q9", phi_var=0.0, tile_rows=rows)
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    J = s.forward(gamma, knots)
    E, V = s.objective_terms()
    s.close()
    _, Eo, _ = oracle_terms(w, gamma, knots)
    assert J == E and abs(E - Eo) <= 1e-10 * abs(Eo) and np.isnan(V)
