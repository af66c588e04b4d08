"""Pins of the oracle's second objective J2 = F_L + w_D F_D + w_T T (Eq. objective2, the oar of Sec. 4.2) and of the
adjoint with it.

Per-step integrands against what the mechanics fixes:
- A uniform flow past a body at rest is seen unchanged on the design grid (the weights sum to one over the
  analysis lattice), so F_L is the design's total kappa^ref times the flow.
- Fluid that moves rigidly with the body exerts no Brinkman force (the hat reproduces linear fields), so all three
  terms vanish at any angle.
- A body spinning in still fluid does the torque work -omega^2 sum kappa^ref |xi - xi^G|^2 / (2 pi l_m |D|)
  (complex-number form).
- A body translating vertically in still fluid does the drag work -V^2 sum kappa^ref / ((x_2^max - x_2^min) |D|).
The adjoint with J2 against complex-step JVPs and central differences, translating and rotating bodies.
"""

import numpy as np
import pytest

import oracle as O
import oracle.lks_oracle as L


def oar_problem(name="D2Q9", kernel="linear", **kw):
    if name == "D2Q9":
        args = dict(shape=(30, 28), periodic=(False, False), design=(6, 4))
    else:
        args = dict(shape=(16, 15, 12), periodic=(False, False, False), design=(4, 3, 2))
    args.update(lattice=name, nu=0.04, kernel=kernel, kappa_max=2.0, Nt=10, K=4, R_t=5.0, R_w=5.0, filter_R=1.6,
                beta=4.0, probe_lo=(2,) * (len(args["shape"])), probe_hi=(4,) * (len(args["shape"])),
                direction=(1.0,) + (0.0,) * (len(args["shape"]) - 1), objective="J2", w_D=0.3, w_T=0.7,
                drag_span=9.0, l_m=3.5)
    args.update(kw)
    return O.Problem(**args)


def body(P, seed):
    kref = O.embed_margin(np.random.default_rng(seed).uniform(0.0, 2.0, P.design), P.margin)
    xg = (np.asarray(P.shape) - 1) / 2 + 0.37
    o = xg - (np.asarray(P.ext) - 1) / 2
    return kref, o, xg


def arms_complex(P):
    XI, ETA = np.meshgrid(np.arange(P.ext[0]), np.arange(P.ext[1]), indexing="ij")
    c = (np.asarray(P.ext) - 1) / 2
    return (XI - c[0]) + 1j * (ETA - c[1])


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("theta", [0.0, 0.8])
def test_uniform_flow_past_a_body_at_rest(kernel, theta):
    P = oar_problem(kernel=kernel)
    kref, o, _ = body(P, 1)
    U = np.array([0.031, -0.012])
    u = np.stack([np.full(P.shape, U[0]), np.full(P.shape, U[1])])
    FL, FD, T = O.oar_terms(P, kref, u, o, theta, 0.0, np.zeros(2))
    assert abs(FL - kref.sum() * U[0] / (P.Nt * np.prod(P.design))) <= 1e-14
    assert FD == 0.0 and T == 0.0


@pytest.mark.parametrize("theta", [0.0, 0.5, -2.2])
def test_fluid_moving_with_the_body_exerts_no_force(theta):
    P = oar_problem()
    kref, o, xg = body(P, 2)
    omega, uG = 0.017, np.array([0.004, -0.009])
    X, Y = np.meshgrid(np.arange(P.shape[0]), np.arange(P.shape[1]), indexing="ij")
    # the rigid velocity field of the body, continued over the whole grid: u^G + omega e_z x (x - x^G)
    u = np.stack([uG[0] - omega * (Y - xg[1]), uG[1] + omega * (X - xg[0])])
    FL, FD, T = O.oar_terms(P, kref, u, o, theta, omega, uG)
    assert max(abs(FL), abs(FD), abs(T)) <= 1e-15


@pytest.mark.parametrize("theta", [0.0, 1.3])
def test_torque_work_of_a_body_spinning_in_still_fluid(theta):
    P = oar_problem()
    kref, o, _ = body(P, 3)
    omega = 0.02
    FL, FD, T = O.oar_terms(P, kref, np.zeros((2,) + P.shape), o, theta, omega, np.zeros(2))
    a = arms_complex(P)
    want = -omega ** 2 * (kref * (a * np.conj(a)).real).sum() / (2 * np.pi * P.l_m * np.prod(P.design))
    assert abs(T - want) <= 1e-13 * abs(want) and FD == 0.0


def test_drag_work_of_a_body_translating_in_still_fluid():
    P = oar_problem()
    kref, o, _ = body(P, 4)
    V = 0.015
    FL, FD, T = O.oar_terms(P, kref, np.zeros((2,) + P.shape), o, 0.4, 0.0, np.array([0.0, V]))
    want = -V ** 2 * kref.sum() / (P.drag_span * np.prod(P.design))
    assert abs(FD - want) <= 1e-13 * abs(want) and abs(FL) <= 1e-16 and T == 0.0


def oar_case(name, kernel, seed, rotate, Nt=10):
    P = oar_problem(name, kernel, Nt=Nt, periodic=(True,) + (False,) * (2 if name == "D3Q15" else 1),
                    **({"shape": (20, 16), "design": (4, 4)} if name == "D2Q9" else {"shape": (14, 13, 9),
                                                                                    "design": (3, 3, 2)}))
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.05, 0.95, P.design)
    knots = rng.normal(0.0, 0.6, (P.K, P.d)) + 0.37
    aknots = rng.normal(0.0, 0.5, 4) + 0.21 if rotate else None
    return P, gamma, knots, aknots


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel,rotate", [("linear", False), ("linear", True), ("cosine", True)])
def test_oar_adjoint_dot_complex_step(name, kernel, rotate):
    P, gamma, knots, aknots = oar_case(name, kernel, 70, rotate)
    res = O.gradient(P, gamma, knots, aknots=aknots)
    J, gg, gk = res[:3]
    rng = np.random.default_rng(71)
    vg, vk = rng.standard_normal(gamma.shape), rng.standard_normal(knots.shape)
    h = 1e-30
    if rotate:
        va = rng.standard_normal(aknots.shape)
        Jc = O.solve(P, gamma + 1j * h * vg, knots + 1j * h * vk, aknots=aknots + 1j * h * va)
        adj = (gg * vg).sum() + (gk * vk).sum() + (res[3] * va).sum()
        scale = np.abs(gg * vg).sum() + np.abs(gk * vk).sum() + np.abs(res[3] * va).sum()
    else:
        Jc = O.solve(P, gamma + 1j * h * vg, knots + 1j * h * vk)
        adj = (gg * vg).sum() + (gk * vk).sum()
        scale = np.abs(gg * vg).sum() + np.abs(gk * vk).sum()
    assert abs(np.real(Jc) - J) <= 1e-12 * abs(J)
    assert abs(adj - np.imag(Jc) / h) <= 1e-12 * scale


def test_oar_adjoint_central_differences():
    P, gamma, knots, aknots = oar_case("D2Q9", "linear", 72, True, Nt=8)
    J, gg, gk, ga = O.gradient(P, gamma, knots, aknots=aknots)
    h = 1e-6
    rng = np.random.default_rng(73)
    for _ in range(2):
        idx = tuple(rng.integers(0, n) for n in gamma.shape)
        gp, gm = gamma.copy(), gamma.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (O.solve(P, gp, knots, aknots=aknots) - O.solve(P, gm, knots, aknots=aknots)) / (2 * h)
        assert abs(fd - gg[idx]) <= 1e-6 * np.max(np.abs(gg)) + 1e-6 * abs(fd)
    for k in range(len(aknots)):
        ap, am = aknots.copy(), aknots.copy()
        ap[k] += h
        am[k] -= h
        fd = (O.solve(P, gamma, knots, aknots=ap) - O.solve(P, gamma, knots, aknots=am)) / (2 * h)
        assert abs(fd - ga[k]) <= 1e-6 * np.max(np.abs(ga)) + 1e-6 * abs(fd)


def test_oar_mistakes_are_caught(monkeypatch):
    test_torque_work_of_a_body_spinning_in_still_fluid(1.3)
    test_drag_work_of_a_body_translating_in_still_fluid()
    orig = L.oar_terms

    def torque_sign_flipped(*a):
        FL, FD, T = orig(*a)
        return FL, FD, -T

    monkeypatch.setattr(O, "oar_terms", torque_sign_flipped)
    with pytest.raises(AssertionError):
        test_torque_work_of_a_body_spinning_in_still_fluid(1.3)
    monkeypatch.setattr(O, "oar_terms", orig)
    # F_D without its u^G_2 weight (plain force instead of work)
    monkeypatch.setattr(O, "oar_terms", lambda P, k, u, o, th, om, uG: orig(P, k, u, o, th, om, uG) if uG[1] == 0
                        else (lambda r: (r[0], r[1] / uG[1], r[2]))(orig(P, k, u, o, th, om, uG)))
    with pytest.raises(AssertionError):
        test_drag_work_of_a_body_translating_in_still_fluid()


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_translating_oar_terms_from_the_mapped_kappa(name, kernel):
    # without rotation, sum_j kappa^ref_j u^ref_j = sum_x kappa_n(x) u_n(x) exactly (both are sum_{x,j} W kappa^ref u),
    # so F_L and F_D follow from the separable mapping of ``map_gather``, a different route from ``oar_terms``'
    # dense transposed mapping
    P = oar_problem(name, kernel, periodic=(True,) + (False,) * (2 if name == "D3Q15" else 1))
    kref, o, _ = body(P, 5)
    rng = np.random.default_rng(6)
    u = rng.normal(0.0, 0.02, (P.d,) + P.shape)
    uG = rng.normal(0.0, 0.01, P.d)
    FL, FD, T = O.oar_terms(P, kref, u, o, 0.0, 0.0, uG)
    kappa, _ = O.map_gather(kref, o, P)
    K = kref.sum()
    nD = np.prod(P.design)
    want_L = ((kappa * u[0]).sum() - uG[0] * K) / (P.Nt * nD)
    want_D = uG[1] * ((kappa * u[1]).sum() - uG[1] * K) / (P.drag_span * nD)
    assert abs(FL - want_L) <= 1e-13 * (abs(want_L) + abs(uG[0] * K) / (P.Nt * nD))
    assert abs(FD - want_D) <= 1e-13 * (abs(want_D) + abs(uG[1] ** 2 * K) / (P.drag_span * nD))
    assert T == 0.0
