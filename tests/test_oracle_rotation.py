"""Pins of the oracle's rotated-body mapping and its adjoint (Sec. 2.3, Eqs. rigid_body_position,
rigid_body_velocity, kappa, u_s; Sec. 2.4, Eqs. psi_filtered, theta, omega; Sec. 2.5, Eq. dJdpsi in discrete form).

- theta = omega = 0 gives the translation mapping (``map_gather``, pinned by brute force elsewhere).
- A quarter and a half turn of the hat-mapped lattice equal numpy's ``rot90`` of kappa^ref.
- The hat and cosine weights sum to one over the analysis lattice, so the mapped kappa and u^S keep the design
  grid's totals at any angle; the hat also reproduces linear functions, so the first moment of kappa is the
  design's first moment turned by e^{i theta} (complex-number form of the rotation), and the mapped velocity's
  angular moment is omega sum_j |xi_j - xi^G|^2 (rigid rotation, counter-clockwise for omega > 0).
- The mapping's derivatives match complex-step derivatives; the full adjoint with angle knots matches a
  complex-step JVP and central differences.
"""
import numpy as np
import pytest

import oracle as O


def problem(name="D2Q9", kernel="linear", periodic=None, shape=None, design=None, **kw):
    if name == "D2Q9":
        shape = shape or (22, 20)
        design = design or (5, 5)
        periodic = periodic if periodic is not None else (True, True)
        probe = dict(probe_lo=(15, 3), probe_hi=(20, 12), direction=(1.0, 0.3))
    else:
        shape = shape or (16, 15, 9)
        design = design or (3, 3, 2)
        periodic = periodic if periodic is not None else (True, True, True)
        probe = dict(probe_lo=(11, 3, 2), probe_hi=(14, 9, 6), direction=(1.0, 0.0, 0.5))
    args = dict(lattice=name, shape=shape, periodic=periodic, nu=0.04, design=design, kernel=kernel, kappa_max=2.0,
                Nt=16, K=4, R_t=6.0, R_w=6.0, filter_R=1.6, beta=4.0, **probe)
    args.update(kw)
    return O.Problem(**args)


def random_kref(P, seed):
    return np.random.default_rng(seed).uniform(0.0, 2.0, P.ext)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_zero_angle_is_the_translation_mapping(name, kernel):
    P = problem(name, kernel, periodic=(True,) + (False,) * (2 if name == "D3Q15" else 1))
    kref = random_kref(P, 1)
    rng = np.random.default_rng(2)
    for _ in range(3):
        # offsets that put part of the body across the periodic seam of x
        o = P.origin() + rng.uniform(-3.0, 3.0, P.d) + np.r_[P.shape[0] / 2 - 2.2, np.zeros(P.d - 1)]
        uG = rng.normal(size=P.d)
        k0, C0 = O.map_gather(kref, o, P)
        k1, uS1 = O.map_rotated(kref, o, 0.0, 0.0, uG, P)
        assert np.max(np.abs(k1 - k0)) <= 1e-13 * np.max(np.abs(k0))
        for a in range(P.d):
            assert np.max(np.abs(uS1[a] - uG[a] * C0)) <= 1e-13 * np.max(np.abs(uG[a] * C0)) + 1e-15


def place(P, arr, center):
    """Analysis-grid field holding `arr` with its centre element at the integer node `center`."""
    out = np.zeros(P.shape)
    lo = [int(center[a]) - (arr.shape[a] - 1) // 2 for a in range(P.d)]
    out[tuple(slice(l, l + n) for l, n in zip(lo, arr.shape))] = arr
    return out


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_quarter_turns_of_the_hat_lattice_are_rot90(turns):
    # odd extended extents put xi^G on a lattice node; an integer x^G then maps every node onto a node
    P = problem("D2Q9", "linear", design=(5, 7), periodic=(False, False), shape=(24, 24))
    kref = random_kref(P, 3)
    o = np.array([11.0, 12.0]) - (np.asarray(P.ext) - 1) / 2  # x^G = (11, 12)
    k, uS = O.map_rotated(kref, o, turns * np.pi / 2, 0.0, np.zeros(2), P)
    want = place(P, np.rot90(kref, k=turns, axes=(0, 1)), (11, 12))
    assert np.max(np.abs(k - want)) <= 1e-12


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_mapped_totals_are_kept_at_any_angle(name, kernel):
    P = problem(name, kernel)
    kref = random_kref(P, 4)
    rng = np.random.default_rng(5)
    for theta in (0.3, -1.1, 2.6):
        o = P.origin() + rng.uniform(-2.0, 2.0, P.d)
        uG, omega = rng.normal(size=P.d), rng.normal()
        k, uS = O.map_rotated(kref, o, theta, omega, uG, P)
        assert abs(k.sum() - kref.sum()) <= 1e-12 * kref.sum()
        nd = kref.size
        for a in range(P.d):  # the design arms sum to zero, so the rotation part carries no net momentum
            assert abs(uS[a].sum() - nd * uG[a]) <= 1e-11 * nd * (abs(uG[a]) + abs(omega))


def hat_problem_inside():
    # walls far from the body, no periodic images: every footprint lies on the grid
    return problem("D2Q9", "linear", periodic=(False, False), shape=(30, 28), design=(6, 4))


@pytest.mark.parametrize("theta", [0.4, 1.9, -2.3])
def test_first_moment_turns_by_exp_i_theta(theta):
    P = hat_problem_inside()
    kref = random_kref(P, 6)
    o = np.array([15.3, 13.6]) - (np.asarray(P.ext) - 1) / 2
    xg = o + (np.asarray(P.ext) - 1) / 2
    k, _ = O.map_rotated(kref, o, theta, 0.0, np.zeros(2), P)
    X, Y = np.meshgrid(np.arange(P.shape[0]), np.arange(P.shape[1]), indexing="ij")
    z_mapped = ((X + 1j * Y) * k).sum() - (xg[0] + 1j * xg[1]) * k.sum()
    XI, ETA = np.meshgrid(np.arange(P.ext[0]), np.arange(P.ext[1]), indexing="ij")
    c = (np.asarray(P.ext) - 1) / 2
    z_design = (((XI - c[0]) + 1j * (ETA - c[1])) * kref).sum()
    assert abs(z_mapped - np.exp(1j * theta) * z_design) <= 1e-11 * abs(z_design)


@pytest.mark.parametrize("theta", [0.0, 0.7, -2.0])
def test_mapped_velocity_is_a_rigid_rotation(theta):
    P = hat_problem_inside()
    o = np.array([14.4, 13.2]) - (np.asarray(P.ext) - 1) / 2
    xg = o + (np.asarray(P.ext) - 1) / 2
    omega = 0.013
    _, uS = O.map_rotated(np.zeros(P.ext), o, theta, omega, np.zeros(2), P)
    X, Y = np.meshgrid(np.arange(P.shape[0]), np.arange(P.shape[1]), indexing="ij")
    ang = ((X - xg[0]) * uS[1] - (Y - xg[1]) * uS[0]).sum()  # z component of sum (x - x^G) x u^S
    XI, ETA = np.meshgrid(np.arange(P.ext[0]), np.arange(P.ext[1]), indexing="ij")
    c = (np.asarray(P.ext) - 1) / 2
    want = omega * ((XI - c[0]) ** 2 + (ETA - c[1]) ** 2).sum()
    assert abs(ang - want) <= 1e-11 * abs(want)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_mapping_derivatives_match_complex_step(name, kernel):
    P = problem(name, kernel, periodic=(True, False) if name == "D2Q9" else (True, False, False))
    kref = random_kref(P, 7)
    rng = np.random.default_rng(8)
    o = P.origin() + rng.uniform(-1.5, 1.5, P.d) + 0.137
    theta, omega, uG = 0.61, 0.021, rng.normal(size=P.d) * 0.01
    _, _, G = O.map_rotated(kref, o, theta, omega, uG, P, with_grad=True)
    h = 1e-30
    kt, ut = O.map_rotated(kref, o, theta + 1j * h, omega, uG, P)
    assert np.max(np.abs(np.imag(kt) / h - G["dk_dth"])) <= 1e-12 * np.max(np.abs(G["dk_dth"]))
    for b in range(P.d):
        ref = np.imag(ut[b]) / h
        assert np.max(np.abs(ref - G["duS_dth"][b])) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300)
    _, uw = O.map_rotated(kref, o, theta, omega + 1j * h, uG, P)
    for b in range(P.d):
        ref = np.imag(uw[b]) / h
        assert np.max(np.abs(ref - G["duS_dom"][b])) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300)
    for a in range(P.d):
        e = np.zeros(P.d, dtype=complex)
        e[a] = 1j * h
        ko, uo = O.map_rotated(kref, o + e, theta, omega, uG, P)
        assert np.max(np.abs(np.imag(ko) / h - G["dk_do"][a])) <= 1e-12 * np.max(np.abs(G["dk_do"][a]))
        for b in range(P.d):
            ref = np.imag(uo[b]) / h
            assert np.max(np.abs(ref - G["duS_do"][a][b])) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300)


def rotating_case(name, kernel, seed, Nt=14):
    if name == "D2Q9":
        P = problem(name, kernel, periodic=(True, False), shape=(20, 16), design=(4, 4), Nt=Nt, K=4,
                    wall_velocity={(1, 1): (0.01, 0.0)}, probe_lo=(13, 0), probe_hi=(18, 9), direction=(1.0, 0.4))
    else:
        P = problem(name, kernel, periodic=(True, False, False), shape=(14, 13, 9), design=(3, 3, 2), Nt=Nt, K=4,
                    probe_lo=(10, 2, 2), probe_hi=(13, 8, 7), direction=(1.0, 0.0, 0.5))
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.05, 0.95, P.design)
    knots = rng.normal(0.0, 0.6, (P.K, P.d)) + 0.37
    aknots = rng.normal(0.0, 0.5, 4) + 0.21
    return P, gamma, knots, aknots


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_rotating_adjoint_dot_complex_step(name, kernel):
    P, gamma, knots, aknots = rotating_case(name, kernel, 60)
    J, gg, gk, ga = O.gradient(P, gamma, knots, aknots=aknots)
    rng = np.random.default_rng(61)
    vg, vk, va = rng.standard_normal(gamma.shape), rng.standard_normal(knots.shape), rng.standard_normal(aknots.shape)
    h = 1e-30
    Jc = O.solve(P, gamma + 1j * h * vg, knots + 1j * h * vk, aknots=aknots + 1j * h * va)
    assert abs(np.real(Jc) - J) <= 1e-12 * abs(J)
    adj = (gg * vg).sum() + (gk * vk).sum() + (ga * va).sum()
    scale = np.abs(gg * vg).sum() + np.abs(gk * vk).sum() + np.abs(ga * va).sum()
    assert abs(adj - np.imag(Jc) / h) <= 1e-12 * scale
    assert np.abs(ga * va).sum() > 1e-3 * scale  # the angle knots matter


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
def test_rotating_adjoint_central_differences(name):
    P, gamma, knots, aknots = rotating_case(name, "linear", 62, Nt=12)
    J, gg, gk, ga = O.gradient(P, gamma, knots, aknots=aknots)
    h = 1e-6
    for k in range(len(aknots)):
        ap, am = aknots.copy(), aknots.copy()
        ap[k] += h
        am[k] -= h
        fd = (O.solve(P, gamma, knots, aknots=ap) - O.solve(P, gamma, knots, aknots=am)) / (2 * h)
        assert abs(fd - ga[k]) <= 1e-6 * np.max(np.abs(ga)) + 1e-6 * abs(fd)


def test_phi_var_with_rotation():
    # the variance source and the rotation together (dot test)
    P, gamma, knots, aknots = rotating_case("D2Q9", "linear", 63, Nt=10)
    P = O.Problem(**{**P.__dict__, "phi_var": 30.0})
    J, gg, gk, ga = O.gradient(P, gamma, knots, aknots=aknots)
    rng = np.random.default_rng(64)
    va = rng.standard_normal(aknots.shape)
    h = 1e-30
    jvp = np.imag(O.solve(P, gamma, knots, aknots=aknots + 1j * h * va)) / h
    assert abs((ga * va).sum() - jvp) <= 1e-12 * np.abs(ga * va).sum()
