"""Pins of the grid-separation mapping (Sec. 2.3, Eqs. kappa, u_s, rigid_body_position with theta = 0)."""
import numpy as np
import pytest

import oracle as O


def prob(shape, periodic, design, kernel, margin=2):
    return O.Problem(lattice="D2Q9" if len(shape) == 2 else "D3Q15", shape=shape, periodic=periodic, nu=0.05,
                     design=design, margin=margin, kernel=kernel)


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_partition_of_unity(kernel):
    r = np.linspace(-3.0, 3.0, 1201)
    tot = sum(O.w1(r - k, kernel) for k in range(-6, 7))
    assert np.max(np.abs(tot - 1.0)) < 1e-14


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("shape,periodic,design", [((20, 17), (True, False), (5, 4)), ((12, 11, 10), (True, False, False), (3, 3, 2))])
def test_gather_equals_bruteforce(kernel, shape, periodic, design):
    P = prob(shape, periodic, design, kernel)
    rng = np.random.default_rng(5)
    kref = O.embed_margin(rng.uniform(0, 1, design), P.margin)
    for trial in range(4):
        o = P.origin() + rng.uniform(-3, 3, len(shape))
        if trial == 0:
            o[0] = o[0] - 7.3  # wrap across the periodic seam
        k1, C1 = O.map_gather(kref, o, P)
        k2, C2 = O.map_bruteforce(kref, o, P)
        assert np.max(np.abs(k1 - k2)) < 1e-14
        assert np.max(np.abs(C1 - C2)) < 1e-14


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_total_and_integer_shift(kernel):
    P = prob((30, 26), (True, True), (6, 5), kernel)
    rng = np.random.default_rng(6)
    kref = O.embed_margin(rng.uniform(0, 1, P.design), P.margin)
    o = P.origin() + np.array([0.37, -0.81])
    k0, _ = O.map_gather(kref, o, P)
    # partition of unity: the interior footprint carries the design total
    assert abs(k0.sum() - kref.sum()) < 1e-13
    # shift by an integer vector m: kappa moves by m exactly
    m = np.array([3, -2])
    k1, _ = O.map_gather(kref, o + m, P)
    assert np.max(np.abs(k1 - np.roll(k0, shift=tuple(m), axis=(0, 1)))) < 1e-15


def test_integer_offset_hat_copies_cosine_smooths():
    P = prob((16, 15), (True, False), (4, 3), "linear")
    rng = np.random.default_rng(7)
    kref = O.embed_margin(rng.uniform(0, 1, P.design), P.margin)
    o = np.array([5.0, 4.0])
    k, _ = O.map_gather(kref, o, P)
    ex = P.ext
    assert np.max(np.abs(k[5:5 + ex[0], 4:4 + ex[1]] - kref)) < 1e-16
    assert abs(k.sum() - kref.sum()) < 1e-14
    Pc = prob((16, 15), (True, False), (4, 3), "cosine")
    kc, _ = O.map_gather(kref, o, Pc)
    # the cosine kernel at integer offsets is the [1/4, 1/2, 1/4] smoothing along every axis
    pad = np.zeros((16, 15))
    pad[5:5 + ex[0], 4:4 + ex[1]] = kref
    sm = pad.copy()
    for a in range(2):
        sm = 0.25 * np.roll(sm, 1, a) + 0.5 * sm + 0.25 * np.roll(sm, -1, a)
    assert np.max(np.abs(kc - sm)) < 1e-15


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_transpose_dot(kernel):
    P = prob((18, 16, 9), (True, False, False), (4, 5, 3), kernel)
    rng = np.random.default_rng(8)
    kref = rng.standard_normal(P.ext)
    g = rng.standard_normal(P.shape)
    o = P.origin() + rng.uniform(-2, 2, 3)
    k, _ = O.map_gather(kref, o, P)
    assert abs((k * g).sum() - (kref * O.map_gather_T(g, o, P)).sum()) < 1e-12 * np.abs(k * g).sum()


@pytest.mark.parametrize("kernel", ["linear", "cosine"])
def test_position_derivative_fd(kernel):
    P = prob((20, 18), (True, False), (5, 4), kernel)
    rng = np.random.default_rng(9)
    kref = O.embed_margin(rng.uniform(0, 1, P.design), P.margin)
    o = P.origin() + np.array([0.31, 0.58])
    _, _, dk, dC = O.map_gather(kref, o, P, with_grad=True)
    h = 1e-6
    for a in range(2):
        e = np.zeros(2)
        e[a] = h
        kp, Cp = O.map_gather(kref, o + e, P)
        km, Cm = O.map_gather(kref, o - e, P)
        assert np.max(np.abs((kp - km) / (2 * h) - dk[a])) < 1e-8
        assert np.max(np.abs((Cp - Cm) / (2 * h) - dC[a])) < 1e-8


def test_hat_derivative_convention_at_integer_offset():
    # reading: the position derivative of the hat map is one-sided from the right in the offset
    P = prob((14, 12), (True, False), (3, 3), "linear")
    rng = np.random.default_rng(10)
    kref = O.embed_margin(rng.uniform(0, 1, P.design), P.margin)
    o = np.array([4.0, 3.0])
    _, _, dk, _ = O.map_gather(kref, o, P, with_grad=True)
    h = 1e-7
    kp, _ = O.map_gather(kref, o + np.array([h, 0.0]), P)
    k0, _ = O.map_gather(kref, o, P)
    assert np.max(np.abs((kp - k0) / h - dk[0])) < 1e-7
