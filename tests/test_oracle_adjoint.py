"""Pins of the oracle's exact discrete adjoint (Sec. 2.5, reverse loop of Algorithm 1).

(1) Dot-product test: dJ/d(design) . v equals the forward-mode directional derivative, taken exactly by
    the complex-step method on the oracle's own forward (no finite-difference truncation error).
(2) Central finite differences on tiny grids, away from the hat kernel's kinks.
(3) The objective J1 = E - phi V of Eq. objective1 against numpy's mean and variance of the space-time sample of
    n.u over the fluid nodes of O_target, and (1), (2) repeated with phi != 0 (the adjoint source then depends on
    E and on the local n.u).
"""
import dataclasses

import numpy as np
import pytest

import oracle as O


PHI_V = 40.0  # large enough that the variance term changes the gradient by O(1) at u ~ 1e-2


def tiny(name, kernel, seed, Nt=24, phi_var=0.0, direction=None):
    if name == "D2Q9":
        shape, periodic, design = (16, 12), (True, False), (4, 4)
        lo, hi, n = (10, 0), (14, 8), (1.0, 0.0)  # the box reaches the wall row y = 0 (excluded from O)
        wall = {(1, 1): (0.01, 0.0)}
    else:
        shape, periodic, design = (12, 9, 8), (True, False, False), (3, 3, 2)
        lo, hi, n = (8, 2, 2), (11, 6, 6), (1.0, 0.0, 0.0)
        wall = {}
    P = O.Problem(lattice=name, shape=shape, periodic=periodic, nu=0.04, design=design, Nt=Nt, K=5, R_t=8.0,
                  kernel=kernel, filter_R=1.6, beta=4.0, kappa_max=2.0, probe_lo=lo, probe_hi=hi,
                  direction=direction or n, wall_velocity=wall, phi_var=phi_var)
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.05, 0.95, design)
    knots = rng.normal(0.0, 0.8, (P.K, len(shape))) + 0.37  # keep clear of integer offsets
    return P, gamma, knots


@pytest.mark.parametrize("name", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel,phi_var", [("linear", 0.0), ("cosine", 0.0), ("linear", PHI_V)])
def test_adjoint_dot_complex_step(name, kernel, phi_var):
    P, gamma, knots = tiny(name, kernel, 20, phi_var=phi_var)
    J, gg, gk = O.gradient(P, gamma, knots)
    rng = np.random.default_rng(21)
    vg = rng.standard_normal(gamma.shape)
    vk = rng.standard_normal(knots.shape)
    h = 1e-30
    Jc = O.solve(P, gamma + 1j * h * vg, knots + 1j * h * vk)
    jvp = np.imag(Jc) / h
    assert abs(np.real(Jc) - J) < 1e-12 * abs(J)
    adj = (gg * vg).sum() + (gk * vk).sum()
    assert abs(adj - jvp) < 1e-12 * (np.abs(gg * vg).sum() + np.abs(gk * vk).sum())


@pytest.mark.parametrize("name,phi_var", [("D2Q9", 0.0), ("D3Q15", 0.0), ("D2Q9", PHI_V)])
def test_adjoint_central_fd(name, phi_var):
    P, gamma, knots = tiny(name, "linear", 30, Nt=20, phi_var=phi_var)
    J, gg, gk = O.gradient(P, gamma, knots)
    h = 1e-6
    rng = np.random.default_rng(31)
    for _ in range(3):
        idx = tuple(rng.integers(0, n) for n in gamma.shape)
        gp, gm = gamma.copy(), gamma.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (O.solve(P, gp, knots) - O.solve(P, gm, knots)) / (2 * h)
        assert abs(fd - gg[idx]) <= 1e-6 * np.max(np.abs(gg)) + 1e-6 * abs(fd)
    for _ in range(3):
        idx = (int(rng.integers(0, P.K)), int(rng.integers(0, P.d)))
        kp, km = knots.copy(), knots.copy()
        kp[idx] += h
        km[idx] -= h
        fd = (O.solve(P, gamma, kp) - O.solve(P, gamma, km)) / (2 * h)
        assert abs(fd - gk[idx]) <= 1e-6 * np.max(np.abs(gk)) + 1e-6 * abs(fd)


def fluid_box(P):
    """Fluid nodes of O_target: the probe box without the first and last planes of every walled axis."""
    keep = np.zeros(P.shape, dtype=bool)
    keep[tuple(slice(lo, hi) for lo, hi in zip(P.probe_lo, P.probe_hi))] = True
    for a, per in enumerate(P.periodic):
        if not per:
            idx = [slice(None)] * P.d
            idx[a] = [0, P.shape[a] - 1]
            keep[tuple(idx)] = False
    return keep


@pytest.mark.parametrize("name,direction", [("D2Q9", (0.6, -0.8)), ("D3Q15", (0.0, 0.6, 0.8))])
def test_variance_objective_is_sample_mean_and_variance(name, direction):
    P, gamma, knots = tiny(name, "linear", 40, Nt=16, phi_var=PHI_V, direction=direction)
    J, states = O.solve(P, gamma, knots, store=True)
    keep = fluid_box(P)
    sample = np.concatenate([np.tensordot(np.asarray(direction), u, axes=1)[keep] for _, u in states[1:]])
    assert sample.size == P.Nt * keep.sum() and np.std(sample) > 1e-4
    want = np.mean(sample) - PHI_V * np.var(sample)
    assert abs(J - want) <= 1e-13 * (abs(np.mean(sample)) + PHI_V * np.var(sample))
    # phi = 0 leaves the mean alone
    assert abs(O.solve(dataclasses.replace(P, phi_var=0.0), gamma, knots) - np.mean(sample)) <= 1e-13 * abs(np.mean(sample))
