"""Pins of the oracle's LKS step against closed forms and invariants (Sec. 2.2).

Every check here is fixed by the mathematics of the scheme, not by the oracle itself:
lattice isotropy, the exact shear-wave decay factor, the exact uniform Brinkman relaxation and
the conservation of total pressure and momentum.
"""

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
def test_isotropy(name):
    # Sec. 2.2 weights: sum w = 1, sum w c_a c_b = delta/3, 4th moment = (dd + dd + dd)/9, odd moments 0
    c, w = O.lattice(name)
    d = c.shape[1]
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(d):
        assert abs((w * c[:, a]).sum()) < 1e-15
        for b in range(d):
            assert abs((w * c[:, a] * c[:, b]).sum() - (a == b) / 3.0) < 1e-15
            for g in range(d):
                assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-15
                for e in range(d):
                    want = ((a == b) * (g == e) + (a == g) * (b == e) + (a == e) * (b == g)) / 9.0
                    assert abs((w * c[:, a] * c[:, b] * c[:, g] * c[:, e]).sum() - want) < 1e-15
    # opposite velocities come in pairs
    s = {tuple(v) for v in c}
    assert all(tuple(-v) in s for v in c)


def test_A_limits():
    # A = 3/4 - 9 nu / 2 (Sec. 2.2): A = 0 at nu = 1/6
    assert O.viscosity_A(1.0 / 6.0) == pytest.approx(0.0, abs=1e-16)
    assert O.viscosity_A(0.0) == 0.75


def _uniform(name, shape, rng):
    c, w = O.lattice(name)
    d = len(shape)
    p = np.full(shape, 1.0 / 3.0 + 0.01)
    u = np.stack([np.full(shape, v) for v in rng.uniform(-0.05, 0.05, d)])
    return c, w, p, u


@pytest.mark.parametrize("name,shape", [("D2Q9", (6, 5)), ("D3Q15", (4, 5, 3))])
def test_uniform_state_is_fixed_point(name, shape):
    rng = np.random.default_rng(1)
    c, w, p, u = _uniform(name, shape, rng)
    mask = np.zeros(shape, bool)
    p1, u1 = O.lks_step(p, u, 0.0, 0.0 * u, O.viscosity_A(0.03), c, w, mask, 0 * u)
    assert np.max(np.abs(p1 - p)) < 1e-15
    assert np.max(np.abs(u1 - u)) < 1e-16


def shear_lambda(k, A):
    # exact one-step factor for u_x = U0 sin(k y), derived in closed form from Eqs. p_tmp, u_tmp:
    # u*(y) = 2/3 u + 1/6 (u(y-1) + u(y+1)) + A/9 (G(y-1) - G(y+1)), G = central difference of u
    return 2.0 / 3.0 + np.cos(k) / 3.0 + (2.0 * A / 9.0) * np.sin(k) ** 2


@pytest.mark.parametrize("name,shape", [("D2Q9", (3, 32)), ("D3Q15", (3, 16, 3))])
@pytest.mark.parametrize("nu,m", [(0.02, 1), (0.1, 3), (0.005, 2)])
def test_shear_wave_exact_decay(name, shape, nu, m):
    c, w = O.lattice(name)
    A = O.viscosity_A(nu)
    ny = shape[1]
    k = 2 * np.pi * m / ny
    y = np.arange(ny)
    U0 = 0.01
    u = np.zeros((len(shape),) + shape)
    prof = U0 * np.sin(k * y)
    u[0] = np.broadcast_to(prof.reshape([1, ny] + [1] * (len(shape) - 2)), shape)
    p = np.full(shape, 1.0 / 3.0)
    mask = np.zeros(shape, bool)
    steps = 1000
    for _ in range(steps):
        p, u = O.lks_step(p, u, 0.0, 0.0 * u, A, c, w, mask, 0 * u)
    lam = shear_lambda(k, A)
    want = prof * lam ** steps
    got = u[0].reshape(shape[0], ny, -1)[0, :, 0]
    assert np.max(np.abs(got - want)) <= 1e-13 * U0
    # u_y and p stay fixed up to rounding of the O(1) terms 3p
    assert np.max(np.abs(u[1:])) < 1e-14
    assert np.max(np.abs(p - 1.0 / 3.0)) < 1e-13  # 1000 steps of rounding
    # lambda = 1 - nu k^2 + O(k^4): the viscosity relation A = 3/4 - 9 nu / 2
    kk = 1e-3
    assert (1.0 - shear_lambda(kk, A)) / kk**2 == pytest.approx(nu, rel=1e-5)


@pytest.mark.parametrize("name,shape", [("D2Q9", (5, 4)), ("D3Q15", (3, 4, 2))])
def test_uniform_brinkman_relaxation(name, shape):
    # kappa, u^S uniform on a periodic box: u_n = U + (u_0 - U) (1 + kappa)^-n (Eq. u, uniform u* = u)
    rng = np.random.default_rng(2)
    c, w, p, u = _uniform(name, shape, rng)
    d = len(shape)
    U = rng.uniform(-0.05, 0.05, d)
    kappa = 0.37
    uS = np.stack([np.full(shape, v) for v in U])
    mask = np.zeros(shape, bool)
    u0 = u[(slice(None),) + (0,) * d].copy()
    for n in range(1, 41):
        p, u = O.lks_step(p, u, kappa, uS, O.viscosity_A(0.05), c, w, mask, 0 * u)
        want = U + (u0 - U) * (1.0 + kappa) ** (-n)
        for a in range(d):
            assert np.max(np.abs(u[a] - want[a])) < 1e-15


def _random_problem(name, shape, periodic, seed, wall_u=None):
    design = tuple(max(2, n // 3) for n in shape)
    P = O.Problem(lattice=name, shape=shape, periodic=periodic, nu=0.04, design=design, Nt=25, K=4, R_t=10.0,
                  probe_lo=tuple(1 for _ in shape), probe_hi=tuple(n - 1 for n in shape),
                  direction=(1.0,) + (0.0,) * (len(shape) - 1))
    if wall_u:
        P.wall_velocity = wall_u
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0, 1, design)
    knots = rng.normal(0, 1.0, (P.K, len(shape)))
    return P, gamma, knots


@pytest.mark.parametrize("name,shape,periodic", [
    ("D2Q9", (14, 12), (True, False)),
    ("D3Q15", (10, 9, 8), (True, False, False)),
])
def test_mass_conservation(name, shape, periodic):
    # sum_x p_n = sum_x p_0: the central-difference divergence telescopes; kappa and walls never touch p
    d = len(shape)
    wall = {(1, 1): (0.03,) + (0.0,) * (d - 1)}
    P, gamma, knots = _random_problem(name, shape, periodic, 3, wall)
    kref, _, _ = O.design_to_kref(P, gamma)
    s, uG = O.positions(knots, P.Nt, P.R_t)
    J, states = O.forward(P, kref, s, uG, store=True)
    m0 = states[0][0].sum()
    for p, _ in states[1:]:
        assert abs(p.sum() - m0) <= 1e-12 * abs(m0)


@pytest.mark.parametrize("name,shape", [("D2Q9", (9, 8)), ("D3Q15", (6, 5, 4))])
def test_momentum_conservation_without_body_or_walls(name, shape):
    rng = np.random.default_rng(4)
    c, w = O.lattice(name)
    d = len(shape)
    p = 1.0 / 3.0 + 0.01 * rng.standard_normal(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    mask = np.zeros(shape, bool)
    mom0 = u.reshape(d, -1).sum(1)
    for _ in range(30):
        p, u = O.lks_step(p, u, 0.0, 0.0 * u, O.viscosity_A(0.03), c, w, mask, 0 * u)
        assert np.max(np.abs(u.reshape(d, -1).sum(1) - mom0)) < 1e-14


def equilibrium_moment_gap(equilibrium, name, seed=5):
    """Largest deviation of the equilibrium's moments from their closed forms (Sec. 2.2, Eq. for f_i^eq).

    Derivation.  With f_i = w_i [3p + 3 c.u + (9/2)(c.u)^2 - (3/2) u.u + A c.S.c] and the lattice identities
    sum_i w_i = 1, sum_i w_i c_a c_b = d_ab / 3, sum_i w_i c_a c_b c_g c_e = (d_ab d_ge + d_ag d_be + d_ae d_bg)/9
    and vanishing odd moments (pinned by test_isotropy):
      sum_i f_i       = 3p + (9/2)|u|^2/3 - (3/2)|u|^2 + A tr(S)/3              = 3p + A tr(S)/3,
      sum_i c_a f_i   = u_a,
      sum_i c_a c_b f_i = p d_ab + (9/2)(|u|^2 d_ab + 2 u_a u_b)/9 - (1/2)|u|^2 d_ab + A (tr(S) d_ab + 2 S_ab)/9
                        = p d_ab + u_a u_b + A (tr(S) d_ab + 2 S_ab)/9.
    The u_a u_b term is the Euler momentum flux of the Navier-Stokes-Brinkman model (Sec. 2.1); it fixes the
    absolute scale of the quadratic terms, which the uniform fixed point (a ratio) and every linear pin (Couette,
    shear wave, channel) leave free.  S_ab = du_b/dx_a + du_a/dx_b is taken from a velocity field linear in space,
    u(x) = U + M x, whose central differences are exact away from the periodic seam: S = M + M^T at the interior
    nodes, known without differencing anything.  p and U are random per case.
    """
    rng = np.random.default_rng(seed)
    c, w = O.lattice(name)
    d = c.shape[1]
    shape = (7,) * d
    worst = 0.0
    for A in (0.0, O.viscosity_A(0.02), O.viscosity_A(0.005)):
        U = rng.uniform(-0.1, 0.1, d)
        M = rng.uniform(-0.01, 0.01, (d, d))  # u_b(x) = U_b + sum_a M[b, a] x_a, so du_b/dx_a = M[b, a]
        X = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
        u = np.stack([U[b] + sum(M[b, a] * X[a] for a in range(d)) for b in range(d)])
        p = 1.0 / 3.0 + 0.02 * rng.standard_normal(shape)
        feq = equilibrium(p, u, A, c, w)
        S = M + M.T  # S[a, b] = du_b/dx_a + du_a/dx_b
        inner = tuple(slice(1, n - 1) for n in shape)
        f = [fi[inner] for fi in feq]
        pi, ui = p[inner], u[(slice(None),) + inner]
        m0 = sum(f)
        worst = max(worst, np.max(np.abs(m0 - (3.0 * pi + A * np.trace(S) / 3.0))))
        for a in range(d):
            m1 = sum(c[i, a] * f[i] for i in range(len(w)))
            worst = max(worst, np.max(np.abs(m1 - ui[a])))
            for b in range(d):
                m2 = sum(c[i, a] * c[i, b] * f[i] for i in range(len(w)))
                want = pi * (a == b) + ui[a] * ui[b] + A * (np.trace(S) * (a == b) + 2.0 * S[a, b]) / 9.0
                worst = max(worst, np.max(np.abs(m2 - want)))
    return worst


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
def test_equilibrium_moments_closed_form(name):
    # zeroth, first and second moments of f^eq against the closed forms derived from the isotropy identities;
    # A = 0 isolates the quadratic terms, A != 0 adds the velocity-gradient term
    assert equilibrium_moment_gap(O.equilibrium, name) < 1e-15
