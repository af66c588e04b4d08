"""Pins of the shape and motion filters (Sec. 3.1 Eqs. filtering, projection; Sec. 2.4 Eq. chi_filtered; Eq. kappa_ref)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


@pytest.mark.parametrize("R", [1.5, 2.0, 2.7])
@pytest.mark.parametrize("shape", [(7, 6), (5, 4, 6)])
def test_density_filter_preserves_constants_and_transpose(R, shape):
    rng = np.random.default_rng(11)
    ones = np.ones(shape)
    assert np.max(np.abs(O.density_filter(0.4 * ones, R) - 0.4)) < 1e-15
    g = rng.uniform(0, 1, shape)
    h = rng.standard_normal(shape)
    lhs = (O.density_filter(g, R) * h).sum()
    rhs = (g * O.density_filter_T(h, R)).sum()
    assert abs(lhs - rhs) < 1e-13 * np.abs(h).sum()
    # against the dense matrix of Eq. filtering
    Wm = O.filter_weights(shape, R)
    dense = (Wm @ g.reshape(-1)) / Wm.sum(1)
    assert np.max(np.abs(dense.reshape(shape) - O.density_filter(g, R))) < 1e-14


def test_density_filter_golden_3x3():
    # hand-computed example, see tests/golden/density_filter_3x3.txt
    gam = np.zeros((3, 3))
    gam[1, 1] = 1.0
    want = load_golden("density_filter_3x3.txt")
    got = O.density_filter(gam, 1.5)
    assert np.max(np.abs(got - want)) < 1e-12


def test_projection_values():
    x = np.linspace(0, 1, 11)
    for beta in (1.0, 8.0, 32.0):
        y = O.projection(x, beta, 0.5)
        assert abs(y[0]) < 1e-15 and abs(y[-1] - 1.0) < 1e-15 and abs(y[5] - 0.5) < 1e-15
        assert np.all(np.diff(y) > 0)
        h = 1e-6
        fd = (O.projection(x + h, beta, 0.5) - O.projection(x - h, beta, 0.5)) / (2 * h)
        assert np.max(np.abs(fd - O.projection_deriv(x, beta, 0.5))) < 1e-6 * beta
    # beta -> 0 tends to the identity
    assert np.max(np.abs(O.projection(x, 1e-5, 0.3) - x)) < 1e-9
    assert np.max(np.abs(O.projection(x, 0.0, 0.3) - x)) == 0.0


def test_kappa_ref():
    assert O.kappa_ref(0.0, 7.0, 0.1) == 0.0
    assert O.kappa_ref(1.0, 7.0, 0.1) == pytest.approx(7.0, rel=1e-15)
    x = np.linspace(0, 1, 9)
    h = 1e-6
    fd = (O.kappa_ref(x + h, 3.0, 0.1) - O.kappa_ref(x - h, 3.0, 0.1)) / (2 * h)
    assert np.max(np.abs(fd - O.kappa_ref_deriv(x, 3.0, 0.1))) < 1e-6


def test_motion_chain():
    rng = np.random.default_rng(12)
    K, Nt, R_t = 9, 80, 25.0
    kn = rng.standard_normal((K, 2))
    # constants are kept by the normalised temporal filter
    assert np.max(np.abs(O.motion_filter(np.full((K, 2), 0.7), Nt, R_t) - 0.7)) < 1e-15
    # a linear motion is kept by the symmetric filter away from the ends
    lin = np.stack([np.arange(K) * 0.5, -np.arange(K) * 0.25], 1)
    f = O.motion_filter(lin, Nt, R_t)
    tk = O.knot_times(K, Nt)
    inner = (tk >= R_t) & (tk <= Nt - R_t)
    assert np.max(np.abs(f[inner] - lin[inner])) < 1e-13
    # interpolation is exact at the knots (integer-only segment index)
    M = O.interp_matrix(K, Nt)
    s = M @ kn
    for k in range(K):
        n = k * Nt // (K - 1)
        if n * (K - 1) == k * Nt:
            assert np.max(np.abs(s[n] - kn[k])) < 1e-15
    # the knot gradient is the transpose of the positions map
    gs = rng.standard_normal((Nt + 1, 2))
    gu = rng.standard_normal((Nt + 1, 2))
    gu[0] = 0.0
    sp, up = O.positions(kn, Nt, R_t)
    P = O.Problem(lattice="D2Q9", shape=(4, 4), periodic=(True, True), nu=0.1, design=(1, 1), Nt=Nt, K=K, R_t=R_t)
    gk = O.knot_gradient(P, gs, gu)
    lhs = (sp * gs).sum() + (up[1:] * gu[1:]).sum()
    assert abs(lhs - (kn * gk).sum()) < 1e-12 * (np.abs(sp * gs).sum() + np.abs(up * gu).sum())
