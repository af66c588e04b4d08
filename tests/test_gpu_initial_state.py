"""lks_set_initial_state (the warm start of the periodic approximation, Sec. 3.3) against the FP64 oracle started
from the same state: a perturbed start, the final state of one forward as the next start, and the reset."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_problem, oracle_run, rel_l2, rel_max, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu
TOL = 1e-10


def check(g, o):
    assert abs(g["J"] - o["J"]) <= TOL * abs(o["J"])
    assert rel_max(g["p"], o["p"]) <= TOL and rel_max(g["u"], o["u"]) <= TOL
    assert rel_l2(g["dgamma"], o["dgamma"]) <= TOL and rel_l2(g["dknots"], o["dknots"]) <= TOL


def run(s, gamma, knots):
    J = s.forward(gamma, knots)
    p, u = s.state()
    dg, dk = s.adjoint()
    return dict(J=J, p=p, u=u, dgamma=dg, dknots=dk)


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
def test_initial_state_matches_oracle(lattice):
    w = tiny_workload(lattice, precision="fp64", Nt=30)
    gamma, knots = draw_gamma(w), draw_knots(w)
    p0, u0 = O.initial_state(oracle_problem(w))
    rng = np.random.default_rng(7)
    p0 = p0 + 1e-3 * rng.standard_normal(p0.shape)
    u0 = u0 + 1e-2 * rng.standard_normal(u0.shape)
    s = Solver.from_workload(w)
    s.set_initial_state(p0, u0)
    g = run(s, gamma, knots)
    o = oracle_run(w, gamma, knots, state0=(p0, u0))
    check(g, o)
    # warm start: the final state of that forward starts the next one
    s.set_initial_state(g["p"], g["u"])
    check(run(s, gamma, knots), oracle_run(w, gamma, knots, state0=(o["p"], o["u"])))
    # reset to the default start
    s.set_initial_state()
    check(run(s, gamma, knots), oracle_run(w, gamma, knots))
    s.close()


@pytest.mark.parametrize("lattice,prec,ckpt", [("D2Q9", "fp64", "full"), ("D3Q15", "fp64", "revolve"),
                                               ("D2Q9", "fp32", "sqrt"), ("D3Q15", "fp32", "sqrt")])
def test_adjoint_terminal_and_initial_state(lattice, prec, ckpt):
    # the adjoint half of the periodic approximation: a terminal adjoint state in, lambda_0 out, against the oracle's
    # adjoint(terminal=..., lambda0=...); then lambda_0 of one run as the terminal state of the next, and the reset
    tol = TOL if prec == "fp64" else 1e-3
    w = tiny_workload(lattice, precision=prec, Nt=24, ckpt=ckpt, ckpt_slots=2, seg_len=5)
    gamma, knots = draw_gamma(w), draw_knots(w)
    P = oracle_problem(w)
    rng = np.random.default_rng(8)
    lp = 1e-4 * rng.standard_normal(P.shape)
    lu = 1e-4 * rng.standard_normal((P.d,) + P.shape)
    s = Solver.from_workload(w)

    def gpu(term):
        s.set_adjoint_terminal(*term) if term is not None else s.set_adjoint_terminal()
        J = s.forward(gamma, knots)
        dg, dk = s.adjoint()
        return dict(J=J, dgamma=dg, dknots=dk, lam0=s.adjoint_initial())

    def same(g, o):
        assert rel_l2(g["dgamma"], o["dgamma"]) <= tol and rel_l2(g["dknots"], o["dknots"]) <= tol
        assert rel_max(g["lam0"][0], o["lam0"][0]) <= tol and rel_max(g["lam0"][1], o["lam0"][1]) <= tol

    g1 = gpu((lp, lu))
    o1 = oracle_run(w, gamma, knots, terminal=(lp, lu))
    same(g1, o1)
    # the terminal state changes the gradient (it is not a no-op)
    assert rel_l2(o1["dgamma"], oracle_run(w, gamma, knots)["dgamma"]) > 1e-3
    # periodic approximation: lambda_0 of this run ends the next reverse sweep
    g2 = gpu(g1["lam0"])
    same(g2, oracle_run(w, gamma, knots, terminal=o1["lam0"]))
    # removed again
    same(gpu(None), oracle_run(w, gamma, knots))
    s.close()
