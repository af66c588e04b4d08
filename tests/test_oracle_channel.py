"""Wall and Brinkman pins: Couette and Brinkman-driven channel steady states (Sec. 2.2, Eqs. p_tmp-u).

For a unidirectional flow u_x(y) every nonlinear term of the LKS step cancels (+-c_x symmetry), p stays
constant and u_y stays zero, so the exact discrete steady state solves a small banded linear system.
That system is derived here by hand from Eqs. p_tmp and u_tmp for one row of nodes:
    u*(y) = 2/3 u(y) + 1/6 (u(y-1) + u(y+1)) + A/9 (G(y-1) - G(y+1)),  G(y) = (u(y+1) - u(y-1)) / 2,
with periodic row indices (walls are the imposed first/last rows) and u = (u* + kappa U)/(1 + kappa)
off the walls.  It is solved directly and compared with the oracle marched to steady state.
"""
import numpy as np
import pytest

import oracle as O


def steady_rows(ny, A, kappa, U, u_lo, u_hi):
    n = ny
    L = np.zeros((n, n))
    for y in range(n):
        # u*(y) as a linear map of the row vector u
        L[y, y] += 2.0 / 3.0
        L[y, (y - 1) % n] += 1.0 / 6.0
        L[y, (y + 1) % n] += 1.0 / 6.0
        # + A/9 G(y-1): G(y-1) = (u(y) - u(y-2))/2
        L[y, y % n] += A / 18.0
        L[y, (y - 2) % n] -= A / 18.0
        # - A/9 G(y+1): G(y+1) = (u(y+2) - u(y))/2
        L[y, (y + 2) % n] -= A / 18.0
        L[y, y % n] += A / 18.0
    M = np.zeros((n, n))
    rhs = np.zeros(n)
    for y in range(n):
        if y == 0 or y == n - 1:
            M[y, y] = 1.0
            rhs[y] = u_lo if y == 0 else u_hi
        else:
            M[y] = -L[y]
            M[y, y] += 1.0 + kappa
            rhs[y] = kappa * U
    return np.linalg.solve(M, rhs)


def march(name, shape, nu, kappa, U, u_hi, steps):
    d = len(shape)
    c, w = O.lattice(name)
    A = O.viscosity_A(nu)
    P = O.Problem(lattice=name, shape=shape, periodic=(True, False) + (True,) * (d - 2), nu=nu, design=(1,) * d,
                  wall_velocity={(1, 1): (u_hi,) + (0.0,) * (d - 1)})
    mask, uw = O.wall_mask(P)
    p, u = O.initial_state(P)
    uS = np.zeros((d,) + shape)
    uS[0] = U
    kap = np.full(shape, kappa)
    for _ in range(steps):
        p, u = O.lks_step(p, u, kap, uS, A, c, w, mask, uw)
    return p, u, A


@pytest.mark.parametrize("name,shape", [("D2Q9", (3, 14)), ("D3Q15", (2, 12, 2))])
def test_couette_discrete_steady_state(name, shape):
    nu, Uw = 0.1, 0.02
    p, u, A = march(name, shape, nu, 0.0, 0.0, Uw, 6000)
    ny = shape[1]
    want = steady_rows(ny, A, 0.0, 0.0, 0.0, Uw)
    got = u[0].reshape(shape[0], ny, -1)[0, :, 0]
    assert np.max(np.abs(got - want)) < 1e-10 * Uw
    assert np.max(np.abs(u[1:])) < 1e-14
    # continuum Couette is linear between the walls; the discrete profile differs by a wall-slip error
    y = np.arange(ny)
    lin = Uw * y / (ny - 1)
    assert np.max(np.abs(got - lin)) < 0.25 * Uw


@pytest.mark.parametrize("name,shape", [("D2Q9", (3, 16)), ("D3Q15", (2, 14, 2))])
def test_brinkman_channel_discrete_steady_state(name, shape):
    nu, kappa, U = 0.05, 0.01, 0.05
    p, u, A = march(name, shape, nu, kappa, U, 0.0, 4000)
    ny = shape[1]
    want = steady_rows(ny, A, kappa, U, 0.0, 0.0)
    got = u[0].reshape(shape[0], ny, -1)[0, :, 0]
    assert np.max(np.abs(got - want)) < 1e-10 * U
    # continuum: U [1 - cosh(m y') / cosh(m h)], m^2 = kappa / nu, walls at distance h from the centre
    h = (ny - 1) / 2.0
    yc = np.arange(ny) - h
    m = np.sqrt(kappa / nu)
    cont = U * (1.0 - np.cosh(m * yc) / np.cosh(m * h))
    # O(dx) wall-slip error of the imposed-velocity walls; bounded loosely, reported by the size of the gap
    assert np.max(np.abs(got - cont)) < 0.3 * U
    # the viscosity coefficient matters: a wrong A moves the profile
    other = steady_rows(ny, A + 0.05, kappa, U, 0.0, 0.0)
    assert np.max(np.abs(got - other)) > 1e-6 * U
