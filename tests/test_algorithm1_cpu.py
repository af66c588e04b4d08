"""The Algorithm 1 driver (beta continuation, stopping rule, volume constraints) on the CPU: with model evaluators,
and with the FP64 oracle's forward and adjoint as the evaluator on a tiny problem."""
import dataclasses

import numpy as np

import oracle as O
from paper_2608_01071_b300.algorithm1 import Settings, run, volume_constraints
from test_oracle_adjoint import tiny


class Quadratic:
    """J = -|gamma - T|^2 - |knots - K0|^2 (maximised), recording the betas it was asked for."""

    def __init__(self, T, K0):
        self.T, self.K0, self.betas = T, K0, []

    def objective(self, beta, gamma, knots):
        self.betas.append(beta)
        self.x = (gamma, knots)
        return -((gamma - self.T) ** 2).sum() - ((knots - self.K0) ** 2).sum()

    def gradient(self):
        g, k = self.x
        return -2 * (g - self.T), -2 * (k - self.K0)


def test_continuation_order_and_active_solid_volume_constraint():
    rng = np.random.default_rng(1)
    T = rng.uniform(0.4, 0.9, (6, 5))  # the unconstrained optimum holds ~65% solid
    ev = Quadratic(T, np.array([[0.5, -0.2], [1.0, 0.3]]))
    s = Settings(betas=(1.0, 2.0), n_opt=300, gamma_step=0.01, pos_step=0.02, V_max_solid=0.4, tol=0.0)
    gamma, knots, h = run(ev, np.full(T.shape, 0.2), np.zeros((2, 2)), s)
    # every iteration of beta 1 before any of beta 2
    assert ev.betas == [1.0] * 300 + [2.0] * 300
    # the constraint is active at the optimum; fixed normalised steps hold it within a few steps of the bound (one
    # step moves the mean of gamma by at most gamma_step, i.e. G1 by at most 0.01 / 0.4)
    assert max(abs(G[0]) for G in h.G[-50:]) <= 3 * 0.01 / 0.4
    assert abs(volume_constraints(gamma, s)[0][0]) <= 3 * 0.01 / 0.4
    assert np.max(np.abs(knots - ev.K0)) <= 0.05  # the unconstrained part converges
    assert np.all((gamma >= 0) & (gamma <= 1))


class Stalling:
    """J changes by 1e-8 relative after the third call of each beta."""

    def __init__(self):
        self.calls = 0

    def objective(self, beta, gamma, knots):
        self.calls += 1
        return 1.0 + (0.5 if self.calls % 100 < 3 else 0.0) * self.calls + 1e-8 * self.calls

    def gradient(self):
        return np.ones((3, 3)), np.ones((2, 2))


def test_stopping_rule_ends_each_beta_before_the_adjoint():
    ev = Stalling()
    _, _, h = run(ev, np.full((3, 3), 0.5), np.zeros((2, 2)), Settings(betas=(1.0, 2.0), n_opt=50, tol=1e-6))
    assert h.stopped_early == [True, True] and len(h.J) < 100


def test_stopping_rule_waits_for_the_constraints():
    # J stalls at once, but the solid volume stays violated: no early stop
    ev = Stalling()
    _, _, h = run(ev, np.full((3, 3), 0.9), np.zeros((2, 2)),
                  Settings(betas=(1.0,), n_opt=20, tol=1e-6, V_max_solid=0.1, gamma_step=0.001))
    assert h.stopped_early == [False] and len(h.J) == 20


class OracleEvaluator:
    def __init__(self, P):
        self.P = P

    def objective(self, beta, gamma, knots):
        self.res = O.gradient(dataclasses.replace(self.P, beta=beta), gamma, knots)
        return self.res[0]

    def gradient(self):
        return self.res[1], self.res[2]


def test_driver_on_the_oracle_raises_J_and_keeps_the_volume():
    P, gamma, knots = tiny("D2Q9", "linear", 90, Nt=16)
    s = Settings(betas=(1.0, 4.0), n_opt=4, gamma_step=0.05, pos_step=0.2, pos_bound=2.0, V_max_solid=0.6, tol=0.0)
    gamma0 = np.clip(gamma, 0.0, 0.55)  # start inside the volume bound
    g, k, h = run(OracleEvaluator(P), gamma0, knots, s)
    assert h.beta == [1.0] * 4 + [4.0] * 4
    assert h.J[3] > h.J[0]  # ascent within the first beta
    assert max(G[0] for G in h.G) <= 0.05


def test_fluid_volume_constraint_and_minimisation():
    # minimise J = |gamma - T|^2 with T mostly fluid, under G2 <= 0 (Eq. constraint2): G2 = mean(1 - gamma) / 0.7 - 1
    # caps the fluid fraction at 70%.  T alone holds about 85% fluid, so the cap binds and the augmented-Lagrangian
    # term has to hold the design at the constraint
    rng = np.random.default_rng(2)
    T = rng.uniform(0.0, 0.3, (5, 5))
    assert (1.0 - T).mean() / 0.7 - 1.0 > 0.15  # the unconstrained optimum breaks G2

    class Bowl:
        def objective(self, beta, gamma, knots):
            self.g = gamma
            return ((gamma - T) ** 2).sum()

        def gradient(self):
            return 2 * (self.g - T), np.zeros((2, 1))

    s = Settings(betas=(1.0,), n_opt=600, maximize=False, gamma_step=0.01, V_max_fluid=0.7, tol=0.0)
    gamma, _, h = run(Bowl(), np.full(T.shape, 0.9), np.zeros((2, 1)), s)
    assert h.J[-1] < h.J[0]
    G2 = [G[0] for G in h.G]
    # the descent reaches the cap (the constraint becomes active); the multiplier then holds the design on it, with
    # the slow oscillation of a first-order multiplier update around G2 = 0
    assert max(G2) > 0.0
    tail = G2[-200:]
    assert max(abs(g) for g in tail) <= 0.06
    assert abs(np.mean(tail)) <= 0.01
    # the constrained minimiser of |gamma - T|^2 under mean(gamma) = 0.3 is T shifted by a constant
    shift = 0.3 - T.mean()
    assert np.max(np.abs(gamma - np.clip(T + shift, 0.0, 1.0))) <= 0.05


def test_angular_speed_constraint_is_enforced():
    # a model rotating body: omega_n = (M a)_n for angle knots a (M a fixed difference operator), J rewards fast
    # rotation; G3 (Eq. constraint3) must end near its bound, and its gradient chain is the transpose of M
    from paper_2608_01071_b300.algorithm1 import angular_speed_bound

    Nt, Kw = 12, 4
    rng = np.random.default_rng(5)
    M = rng.uniform(0.0, 1.0, (Nt + 1, Kw)) / Kw
    M[0] = 0.0

    class Spinner:
        def objective(self, beta, gamma, knots, aknots):
            self.a = aknots
            self.om = M @ aknots
            return float(self.om[1:].sum())

        def gradient(self):
            return np.zeros((2, 2)), np.zeros((2, 1)), M[1:].sum(axis=0)

        def angles(self):
            return np.cumsum(self.om), self.om

        def angles_T(self, g_theta, g_omega):
            return M.T @ np.asarray(g_omega) + M.T @ np.cumsum(np.asarray(g_theta)[::-1])[::-1]

    # G3 of a constant speed: (Nt |om/om_max|^p)^(1/p) - 1, and its gradient against central differences
    om = np.full(Nt + 1, 0.02)
    G3, g = angular_speed_bound(om, 0.01, 8.0)
    assert abs(G3 - (Nt ** (1 / 8.0) * 2.0 - 1.0)) <= 1e-12
    h = 1e-7
    e = np.zeros(Nt + 1)
    e[3] = h
    fd = (angular_speed_bound(om + e, 0.01, 8.0)[0] - angular_speed_bound(om - e, 0.01, 8.0)[0]) / (2 * h)
    assert abs(fd - g[3]) <= 1e-6 * abs(g[3])
    s = Settings(betas=(1.0,), n_opt=300, omega_max=0.05, p_G3=8.0, ang_step=0.01, tol=0.0)
    _, _, a, h = run(Spinner(), np.full((2, 2), 0.5), np.zeros((2, 1)), s, aknots=np.zeros(Kw))
    G3s = [G[0] for G in h.G]
    assert max(G3s) > 0.0  # the ascent reaches the bound
    # then the multiplier holds omega at the bound: the first-order update settles into a small limit cycle around it
    tail = G3s[-100:]
    assert abs(np.mean(tail)) <= 0.05 and max(tail) <= 0.3
    assert h.J[-1] > h.J[0]
