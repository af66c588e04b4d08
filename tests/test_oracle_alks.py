"""The paper's continuous adjoint (ALKS, Sec. 2.5, Eqs. ap_tmp-as) in the oracle, against the exact discrete adjoint
and finite differences.

- Where the two schemes have the same algebra they must agree: with A = 3/4 - 9 nu / 2 = 0 (nu = 1/6) the ALKS
  differs from the exact adjoint only in the velocity-dependent terms of its equilibrium, which it evaluates one
  node upstream and one step later. The difference therefore vanishes linearly with the flow speed. This checks
  the mapping p~ = -lambda_p / 3, u~ = -lambda_u / (3 (1 + kappa)), the implicit Brinkman update, the objective
  source and the sensitivity forms.
- An Appendix-A-style case (walls on every side, a body moving only vertically with a cosine history,
  kappa_max^ref = 200, nu = 0.1) compares the motion sensitivities. The exact adjoint matches central differences
  to 1e-6. The ALKS, which applies the velocity-gradient term one step later, agrees to within a few percent,
  matching the "slight differences" reported against finite differences.
"""
import numpy as np

import oracle as O


def rl2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def vertical_case(nu, amp, kappa_max=2.0, shape=(40, 36), design=(8, 8), Nt=120, K=7, probe_x=30, seed=0):
    P = O.Problem(lattice="D2Q9", shape=shape, periodic=(False, False), nu=nu, design=design, kappa_max=kappa_max,
                  q=0.1, Nt=Nt, K=K, R_t=Nt / 10, filter_R=0.0, beta=0.0, probe_lo=(probe_x, 4),
                  probe_hi=(probe_x + 1, shape[1] - 4), direction=(1.0, 0.0))
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.05, 0.95, P.design)
    k = np.arange(P.K)
    knots = np.stack([np.zeros(P.K), amp * np.cos(2 * np.pi * k / (P.K - 1))], axis=1) + 0.3
    return P, gamma, knots


def test_alks_equals_the_exact_adjoint_at_A0_to_first_order_in_the_flow_speed():
    errs = []
    for amp in (0.5, 0.05):
        P, gamma, knots = vertical_case(1.0 / 6.0, amp)
        assert O.viscosity_A(P.nu) == 0.0
        J, gg, gk = O.gradient(P, gamma, knots)
        Ja, ga, gka, _, _ = O.gradient_alks(P, gamma, knots)
        assert Ja == J
        errs.append((rl2(ga, gg), rl2(gka, gk)))
    assert errs[1][0] <= 2e-3 and errs[1][1] <= 2e-3
    # ten times the speed, about ten times the difference
    for e_fast, e_slow in zip(errs[0], errs[1]):
        assert 5.0 <= e_fast / e_slow <= 20.0


def test_alks_motion_sensitivity_appendix_a_style():
    P, gamma, knots = vertical_case(0.1, 12.0, kappa_max=200.0, shape=(60, 60), design=(12, 12), Nt=300, K=11,
                                    probe_x=45)
    gamma = (gamma > 0.5) * 0.9 + 0.05  # a nearly binary body
    J, gg, gk = O.gradient(P, gamma, knots)
    _, ga, gka, _, _ = O.gradient_alks(P, gamma, knots)
    # exact adjoint against central differences at the knot of largest sensitivity
    k = int(np.argmax(np.abs(gk[:, 1])))
    h = 1e-6
    kp, km = knots.copy(), knots.copy()
    kp[k, 1] += h
    km[k, 1] -= h
    fd = (O.solve(P, gamma, kp) - O.solve(P, gamma, km)) / (2 * h)
    assert abs(fd - gk[k, 1]) <= 1e-6 * abs(fd)
    # the ALKS motion sensitivity: same shape, a few percent off
    assert rl2(gka[:, 1], gk[:, 1]) <= 0.1
    assert np.corrcoef(gka[:, 1], gk[:, 1])[0, 1] >= 0.99
    assert np.sign(gka[k, 1]) == np.sign(gk[k, 1])
