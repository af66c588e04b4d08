"""Pins of the oracle's parts of Algorithm 1 beyond one forward/adjoint pair: the constraint functionals G1-G3
(Sec. 2.6, Eqs. constraint1-3) and the adjoint's terminal and initial states used by the periodic approximation
(Sec. 3.3).

- G1, G2 of a uniform design and the identity G1 + G2 = 1/V_max - 2; G3 of a constant angular speed, and G3 -> the
  max-norm bound as p grows; their gradients (and G3's chain to the angle knots) by complex step.
- The adjoint with a terminal state L added returns the gradient of J plus that of the linear functional
  <L, (p_Nt, u_Nt)>, and its state at n = 0 is the gradient of J with respect to the initial state; both are checked
  against complex-step derivatives of the forward.
"""

import numpy as np
import pytest

import oracle as O
from test_oracle_adjoint import tiny


def test_volume_constraints():
    rng = np.random.default_rng(1)
    g = np.full((5, 4), 0.3)
    G1, d1 = O.solid_volume(g, 0.6)
    G2, d2 = O.fluid_volume(g, 0.8)
    assert abs(G1 - (0.3 / 0.6 - 1)) <= 1e-15 and abs(G2 - (0.7 / 0.8 - 1)) <= 1e-15
    g = rng.uniform(0, 1, (6, 7))
    assert abs(O.solid_volume(g, 0.5)[0] + O.fluid_volume(g, 0.5)[0] - (1 / 0.5 - 2)) <= 1e-14
    v = rng.standard_normal(g.shape)
    h = 1e-30
    for f in (O.solid_volume, O.fluid_volume):
        jvp = np.imag(f(g + 1j * h * v, 0.7)[0]) / h
        assert abs((f(g, 0.7)[1] * v).sum() - jvp) <= 1e-14 * np.abs(v).sum()


def test_angular_speed_bound():
    Nt, p = 40, 16
    om = np.full(Nt + 1, 0.0007)
    G3, _ = O.angular_speed_bound(om, 0.001, p)
    assert abs(G3 - (Nt ** (1 / p) * 0.7 - 1)) <= 1e-14
    # the p-norm tends to the largest |omega| (numpy's max) as p grows
    om = np.random.default_rng(2).uniform(-0.0009, 0.0009, Nt + 1)
    G3, _ = O.angular_speed_bound(om, 0.001, 4000)
    assert abs((G3 + 1) - np.max(np.abs(om[1:])) / 0.001) <= 2e-3
    # gradient by complex step, then through the angles to the angle knots
    om = np.random.default_rng(3).uniform(-0.0009, 0.0009, Nt + 1)
    v = np.random.default_rng(4).standard_normal(Nt + 1)
    h = 1e-30
    G3, g = O.angular_speed_bound(om, 0.001, p)
    jvp = np.imag(O.angular_speed_bound(om + 1j * h * v, 0.001, p)[0]) / h
    assert abs((g * v).sum() - jvp) <= 1e-12 * np.abs(g * v).sum()
    P = O.Problem(lattice="D2Q9", shape=(8, 8), periodic=(True, True), nu=0.1, design=(2, 2), Nt=Nt, R_w=9.0)
    ak = np.array([0.01, -0.02, 0.015, 0.0])
    va = np.random.default_rng(5).standard_normal(4)
    G3, g = O.angular_speed_bound(O.angles(ak, Nt, P.R_w)[1], 0.001, p)
    ga = O.angle_gradient(P, np.zeros(Nt + 1), g, len(ak))
    jvp = np.imag(O.angular_speed_bound(O.angles(ak + 1j * h * va, Nt, P.R_w)[1], 0.001, p)[0]) / h
    assert abs((ga * va).sum() - jvp) <= 1e-12 * np.abs(ga * va).sum()


def pieces(P, gamma, knots):
    kref, _, _ = O.design_to_kref(P, gamma)
    s, uG = O.positions(knots, P.Nt, P.R_t)
    return kref, s, uG


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
def test_adjoint_terminal_state_adds_the_final_state_functional(name):
    P, gamma, knots = tiny(name, "linear", 80, Nt=12)
    kref, s, uG = pieces(P, gamma, knots)
    rng = np.random.default_rng(81)
    Lp, Lu = rng.standard_normal(P.shape), rng.standard_normal((P.d,) + P.shape)
    _, states = O.forward(P, kref, s, uG, store=True)
    g0 = O.adjoint(P, kref, s, uG, states)[0]
    g1 = O.adjoint(P, kref, s, uG, states, terminal=(Lp, Lu))[0]
    # d/d kref of <L, x_Nt> by complex step along a random direction of kref
    v = rng.standard_normal(kref.shape)
    h = 1e-30
    _, st = O.forward(P, kref + 1j * h * v, s, uG, store=True)
    pN, uN = st[-1]
    jvp = np.imag((Lp * pN).sum() + (Lu * uN).sum()) / h
    assert abs(((g1 - g0) * v).sum() - jvp) <= 1e-11 * np.abs((g1 - g0) * v).sum()


@pytest.mark.parametrize("name,phi_var", [("D2Q9", 0.0), ("D3Q15", 0.0), ("D2Q9", 40.0)])
def test_adjoint_initial_state_is_the_gradient_wrt_the_initial_state(name, phi_var):
    P, gamma, knots = tiny(name, "linear", 82, Nt=12, phi_var=phi_var)
    kref, s, uG = pieces(P, gamma, knots)
    rng = np.random.default_rng(83)
    p0, u0 = O.initial_state(P)
    p0 = p0 + 0.01 * rng.standard_normal(P.shape)
    u0 = u0 + 0.01 * rng.standard_normal(u0.shape)
    _, states = O.forward(P, kref, s, uG, store=True, state0=(p0, u0))
    lam0 = []
    O.adjoint(P, kref, s, uG, states, lambda0=lam0)
    lp, lu = lam0[0]
    vp, vu = rng.standard_normal(P.shape), rng.standard_normal(u0.shape)
    h = 1e-30
    J = O.forward(P, kref, s, uG, state0=(p0 + 1j * h * vp, u0 + 1j * h * vu))
    jvp = np.imag(J) / h
    assert abs((lp * vp).sum() + (lu * vu).sum() - jvp) <= 1e-12 * (np.abs(lp * vp).sum() + np.abs(lu * vu).sum())
