"""Planted mistakes in the oracle (on the CPU) must make its pins fail.

Each test patches one plausible error into the oracle and checks that the corresponding pin catches it,
so a green pin run says something about the oracle's correctness.
"""
import numpy as np
import pytest

import oracle as O
import oracle.lks_oracle as L

from test_oracle_lattice import shear_lambda
from test_oracle_adjoint import tiny


def shear_error(A_used, A_true, name="D2Q9"):
    c, w = O.lattice(name)
    shape = (3, 32)
    k = 2 * np.pi / 32
    prof = 0.01 * np.sin(k * np.arange(32))
    u = np.zeros((2,) + shape)
    u[0] = prof[None, :]
    p = np.full(shape, 1 / 3)
    mask = np.zeros(shape, bool)
    for _ in range(200):
        p, u = O.lks_step(p, u, 0.0, 0 * u, A_used, c, w, mask, 0 * u)
    return np.max(np.abs(u[0, 0] - prof * shear_lambda(k, A_true) ** 200))


def test_wrong_viscosity_coefficient_is_caught():
    nu = 0.02
    assert shear_error(O.viscosity_A(nu), O.viscosity_A(nu)) < 1e-15
    assert shear_error(0.75 - 4.0 * nu, O.viscosity_A(nu)) > 1e-6


def test_wrong_weight_is_caught():
    c, w = O.lattice("D2Q9")
    w2 = w.copy()
    w2[5:] = 1.0 / 30.0
    w2[0] = 1.0 - w2[1:].sum()
    assert abs((w2 * c[:, 0] ** 2).sum() - 1 / 3) > 1e-3


def test_forward_adjoint_mismatch_is_caught(monkeypatch):
    P, gamma, knots = tiny("D2Q9", "linear", 50, Nt=8)
    rng = np.random.default_rng(51)
    vg = rng.standard_normal(gamma.shape)

    def dot_gap():
        J, gg, gk = O.gradient(P, gamma, knots)
        h = 1e-30
        jvp = np.imag(O.solve(P, gamma + 1j * h * vg, knots)) / h
        return abs((gg * vg).sum() - jvp) / np.abs(gg * vg).sum()

    assert dot_gap() < 1e-12
    # a one-sided velocity gradient in the forward only (the adjoint keeps the central transpose)
    monkeypatch.setattr(L, "central_diff", lambda f, axis: np.roll(f, -1, axis=axis) - f)
    assert dot_gap() > 1e-6


def test_dropped_brinkman_term_is_caught(monkeypatch):
    # drop kappa u^S from Eq. u: the uniform relaxation closed form must fail
    c, w = O.lattice("D2Q9")
    shape = (4, 4)
    u = np.zeros((2,) + shape)
    p = np.full(shape, 1 / 3)
    uS = np.full((2,) + shape, 0.05)
    mask = np.zeros(shape, bool)
    orig = L.lks_step

    def bad(p, u, kappa, uS, A, c, w, mask, uw):
        return orig(p, u, kappa, 0.0 * uS, A, c, w, mask, uw)

    monkeypatch.setattr(L, "lks_step", bad)
    p1, u1 = L.lks_step(p, u, 0.5, uS, 0.6, c, w, mask, 0 * u)
    want = 0.05 + (0.0 - 0.05) / 1.5
    assert abs(u1[0, 0, 0] - want) > 1e-3


@pytest.mark.parametrize("mistake", ["drop_mean", "sign"])
def test_variance_source_mistake_is_caught(monkeypatch, mistake):
    from test_oracle_adjoint import PHI_V

    P, gamma, knots = tiny("D2Q9", "linear", 52, Nt=8, phi_var=PHI_V)
    rng = np.random.default_rng(53)
    vg = rng.standard_normal(gamma.shape)

    def dot_gap():
        J, gg, gk = O.gradient(P, gamma, knots)
        h = 1e-30
        jvp = np.imag(O.solve(P, gamma + 1j * h * vg, knots)) / h
        return abs((gg * vg).sum() - jvp) / np.abs(gg * vg).sum()

    assert dot_gap() < 1e-12
    fa = L.flow_along
    if mistake == "drop_mean":  # the 2 phi E term of dJ1/du left out
        bad = lambda prob, phi, E, u: phi * (1.0 - 2.0 * prob.phi_var * fa(prob, u))
    else:  # the variance term with the wrong sign
        bad = lambda prob, phi, E, u: phi * (1.0 - 2.0 * prob.phi_var * E + 2.0 * prob.phi_var * fa(prob, u))
    monkeypatch.setattr(L, "objective_source", bad)
    assert dot_gap() > 1e-6


def test_rotation_mistakes_are_caught(monkeypatch):
    # each plausible slip in the rotated mapping makes one of its pins fail (the pins pass unpatched)
    import test_oracle_rotation as R

    R.test_first_moment_turns_by_exp_i_theta(0.4)
    R.test_mapped_velocity_is_a_rigid_rotation(0.7)
    R.test_mapping_derivatives_match_complex_step("D2Q9", "linear")
    rot, rot_d, rot_dd = L.rotation_matrix, L.rotation_matrix_d, L.rotation_matrix_dd
    # the body turned the wrong way (R^T for R)
    monkeypatch.setattr(L, "rotation_matrix", lambda th: rot(th).T)
    with pytest.raises(AssertionError):
        R.test_first_moment_turns_by_exp_i_theta(0.4)
    monkeypatch.setattr(L, "rotation_matrix", rot)
    # the rigid velocity with the wrong sense of rotation
    monkeypatch.setattr(L, "rotation_matrix_d", lambda th: -rot_d(th))
    with pytest.raises(AssertionError):
        R.test_mapped_velocity_is_a_rigid_rotation(0.7)
    monkeypatch.setattr(L, "rotation_matrix_d", rot_d)
    # d u^S,ref / d theta dropped
    monkeypatch.setattr(L, "rotation_matrix_dd", lambda th: 0.0 * rot_dd(th))
    with pytest.raises(AssertionError):
        R.test_mapping_derivatives_match_complex_step("D2Q9", "linear")


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
def test_doubled_quadratic_terms_are_caught(name):
    # both 1/2 factors of the quadratic terms dropped (9 (c.u)^2 - 3 u.u): the ratio 3 that the uniform fixed
    # point checks is kept, the second moment's Euler flux u_a u_b doubles
    from test_oracle_lattice import equilibrium_moment_gap

    def doubled(p, u, A, c, w):
        feq = O.equilibrium(p, u, A, c, w)
        d = u.shape[0]
        uu = sum(u[a] * u[a] for a in range(d))
        out = []
        for i in range(len(w)):
            cu = sum(c[i, a] * u[a] for a in range(d))
            out.append(feq[i] + w[i] * (4.5 * cu * cu - 1.5 * uu))
        return out

    assert equilibrium_moment_gap(O.equilibrium, name) < 1e-15
    assert equilibrium_moment_gap(doubled, name) > 1e-4
    # the fixed-point pin alone does not see it
    rng = np.random.default_rng(1)
    c, w = O.lattice(name)
    shape = (5, 4) if name == "D2Q9" else (4, 3, 3)
    d = len(shape)
    p = np.full(shape, 1.0 / 3.0 + 0.01)
    u = np.stack([np.full(shape, v) for v in rng.uniform(-0.05, 0.05, d)])
    f = doubled(p, u, 0.5, c, w)
    g = [np.roll(fi, shift=tuple(int(v) for v in c[i]), axis=tuple(range(d))) for i, fi in enumerate(f)]
    ustar = sum(c[i, 0] * g[i] for i in range(len(w)))
    assert np.max(np.abs(ustar - u[0])) < 1e-15
