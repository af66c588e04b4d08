"""The paper's continuous adjoint (ALKS, Sec. 2.5, Eqs. ap_tmp-as) on the CUDA path against the oracle's adjoint_alks,
and beside the exact discrete adjoint.

The ALKS is an approximation of the gradient (its Brinkman source is explicit and its velocity-gradient term lags), so
the reference for its numbers is the oracle's ALKS written from the same equations: J, both gradients and the
per-step motion sensitivities.  Against the exact discrete adjoint on the GPU it agrees closely but not exactly, as
the paper's Appendix A reports for its finite-difference comparison.
"""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_problem, rel_l2, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-3}


def run(w, gamma, knots):
    s = Solver.from_workload(w)
    J = s.forward(gamma, knots)
    dg, dk = s.adjoint()
    gs, gu = s.step_sensitivities()
    s.close()
    return J, dg, dk, gs, gu


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alks_matches_oracle(lattice, kernel, prec):
    w = tiny_workload(lattice, kernel=kernel, precision=prec, adjoint="alks", Nt=30 if lattice == "D2Q9" else 20)
    gamma, knots = draw_gamma(w), draw_knots(w)
    J, dg, dk, gs, gu = run(w, gamma, knots)
    Jo, dgo, dko, gso, guo = O.gradient_alks(oracle_problem(w), gamma, knots)
    tol = TOL[prec]
    assert abs(J - Jo) <= max(tol, 1e-5 if prec == "fp32" else tol) * abs(Jo)
    assert rel_l2(dg, dgo) <= tol and rel_l2(dk, dko) <= tol
    assert rel_l2(gs[1:], gso[1:]) <= tol and rel_l2(gu[1:], guo[1:]) <= tol


@pytest.mark.parametrize("ckpt", ["sqrt", "revolve"])
def test_alks_checkpointed(ckpt):
    w = tiny_workload("D3Q15", precision="fp64", adjoint="alks", Nt=17, ckpt=ckpt, ckpt_slots=2, seg_len=4)
    gamma, knots = draw_gamma(w), draw_knots(w)
    J, dg, dk, gs, gu = run(w, gamma, knots)
    Jo, dgo, dko, gso, guo = O.gradient_alks(oracle_problem(w), gamma, knots)
    assert rel_l2(dg, dgo) <= 1e-10 and rel_l2(dk, dko) <= 1e-10


def test_alks_beside_exact_adjoint():
    # same J (the forward is shared); gradients correlated but not equal (the ALKS is the continuous adjoint)
    w = tiny_workload("D2Q9", precision="fp64", Nt=40)
    gamma, knots = draw_gamma(w), draw_knots(w)
    J1, dg1, dk1, gs1, _ = run(w, gamma, knots)
    J2, dg2, dk2, gs2, _ = run(dict(w, adjoint="alks"), gamma, knots)
    assert J1 == J2
    corr = np.corrcoef(gs1[1:].ravel(), gs2[1:].ravel())[0, 1]
    assert corr > 0.9
    assert rel_l2(dg2, dg1) > 1e-6  # a different adjoint, not a copy of the exact one
