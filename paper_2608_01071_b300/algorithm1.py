"""The optimisation procedure of Algorithm 1 around the solver (Sec. 3.2-3.4).

- beta continuation: for each beta of the schedule, up to N_opt design iterations (Sec. 3.2).
- Stopping rule: after the forward solve of iteration k+1, stop this beta when |J^{k+1} - J^k| / |J^k| <= tol and
  every constraint G_j <= 0 holds (Sec. 3.2). As in Algorithm 1, the check comes before the adjoint solve.
- Volume constraints G1 (solid) and G2 (fluid) of Eqs. constraint1-2, on the design variable gamma.
- With a rotating body (angle knots), the angular-speed constraint G3 of Eq. constraint3 on omega_n, the p-norm
  bound (sum_{n=1..Nt} |omega_n / omega_max|^p)^(1/p) - 1 <= 0 (rectangle rule with unit step, like the objectives);
  omega_n and the chain from d G3 / d omega_n to the angle knots come from the library (lks_get_angles, lks_angles_T).
- Periodic approximation (Sec. 3.3): the final state of one forward solve starts the next, and the adjoint state at
  n = 0 of one reverse sweep ends the next (``SolverEvaluator(periodic=True)``, through lks_get_state /
  lks_set_initial_state and lks_get_adjoint_initial / lks_set_adjoint_terminal).

The paper updates the design with MMA, which is not part of this library. This driver takes normalised
projected-gradient steps on an augmented Lagrangian of the inequality constraints instead.
- Direction: d = grad J / |grad J|_inf - sum_j max(0, rho G_j + mu_j) grad G_j / |grad G_j|_inf, with the sign
  of J flipped when minimising.
- Update: gamma <- clip(gamma + s_g d / |d|_inf, 0, 1) and knots <- clip(knots + s_p d_k / |d_k|_inf, -b, b).
- Move limits: s_g and s_p are kept per variable. One shrinks by 0.7 when its step changes sign from the previous
  iteration (an oscillation) and grows by 1.2, up to the initial limit, when it keeps its sign. This is the move-limit
  rule of MMA's asymptote update in its simplest form. The limits restart with every beta.
- Multipliers: mu_j <- max(0, mu_j + rho G_j) after every iteration.

The driver works on host arrays. The evaluator does the forward and adjoint solves; ``SolverEvaluator`` runs them
through the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Settings:
    betas: tuple = (1.0, 2.0, 4.0, 8.0, 16.0, 32.0)  # projection steepness schedule (Sec. 4)
    n_opt: int = 100                 # iterations per beta at most
    tol: float = 1e-6                # stopping rule |J^{k+1} - J^k| / |J^k| <= tol
    maximize: bool = True
    gamma_step: float = 0.05
    pos_step: float = 0.5            # cells
    pos_bound: float = np.inf        # |knot offset| bound, cells
    V_max_solid: float | None = None  # G1 of Eq. constraint1 (None: not imposed)
    V_max_fluid: float | None = None  # G2 of Eq. constraint2
    omega_max: float | None = None   # G3 of Eq. constraint3 (None: not imposed; needs angle knots)
    p_G3: float = 8.0                # exponent of G3's p-norm
    ang_step: float = 0.01           # angle-knot move limit, radians
    ang_bound: float = np.inf        # |angle knot| bound, radians
    rho: float = 10.0                # augmented-Lagrangian penalty on the normalised constraint directions


def volume_constraints(gamma, s: Settings):
    """[(G_j, dG_j/dgamma)] of the imposed volume constraints (Eqs. constraint1, constraint2; D = the design grid)."""
    n = gamma.size
    out = []
    if s.V_max_solid is not None:
        out.append((gamma.sum() / (s.V_max_solid * n) - 1.0, np.full(gamma.shape, 1.0 / (s.V_max_solid * n))))
    if s.V_max_fluid is not None:
        out.append(((1.0 - gamma).sum() / (s.V_max_fluid * n) - 1.0, np.full(gamma.shape, -1.0 / (s.V_max_fluid * n))))
    return out


def angular_speed_bound(omega, omega_max, p):
    """G3 = (sum_{n>=1} |omega_n / omega_max|^p)^(1/p) - 1 and dG3/domega_n (Eq. constraint3; omega_0 enters no step)."""
    r = np.asarray(omega, dtype=np.float64)[1:] / omega_max
    S = (np.abs(r) ** p).sum()
    g = np.zeros(len(omega))
    if S > 0.0:
        g[1:] = S ** (1.0 / p - 1.0) * np.abs(r) ** (p - 1.0) * np.sign(r) / omega_max
    return S ** (1.0 / p) - 1.0, g


def _unit(a):
    m = np.max(np.abs(a)) if a.size else 0.0
    return a / m if m > 0.0 else np.zeros_like(a)


def _adapt(lim, d, d_prev, top):
    """Per-variable move limits: x0.7 where the step reverses, x1.2 (at most `top`) where it keeps its sign."""
    prod = d * d_prev
    return np.where(prod < 0.0, 0.7 * lim, np.where(prod > 0.0, np.minimum(1.2 * lim, top), lim))


@dataclass
class History:
    beta: list = field(default_factory=list)
    J: list = field(default_factory=list)
    G: list = field(default_factory=list)
    stopped_early: list = field(default_factory=list)  # one flag per beta


def run(evaluator, gamma, knots, s: Settings = Settings(), callback=None, aknots=None):
    """Algorithm 1 from (gamma, knots) and, for a rotating body, the angle knots aknots. Returns (gamma, knots, History),
    or (gamma, knots, aknots, History) with angle knots.

    evaluator.objective(beta, gamma, knots[, aknots]) runs the forward solve and returns J. evaluator.gradient() then
    returns (dJ/dgamma, dJ/dknots[, dJ/daknots]) of that same forward solve. With G3, evaluator.angles() returns
    (theta_n, omega_n) of that forward and evaluator.angles_T(g_theta, g_omega) the chain to the angle knots.
    """
    gamma = np.array(gamma, dtype=np.float64)
    knots = np.array(knots, dtype=np.float64)
    rot = aknots is not None
    if rot:
        aknots = np.array(aknots, dtype=np.float64)
    if s.omega_max is not None and not rot:
        raise ValueError("G3 (omega_max) needs angle knots")
    sign = 1.0 if s.maximize else -1.0
    hist = History()
    mu = None
    for beta in s.betas:
        J_prev = None
        stopped = False
        lim_g = np.full(gamma.shape, s.gamma_step)
        lim_k = np.full(knots.shape, s.pos_step)
        lim_a = np.full(aknots.shape, s.ang_step) if rot else None
        prev_g = prev_k = prev_a = None
        for _ in range(s.n_opt):
            J = evaluator.objective(beta, gamma, knots, aknots) if rot else evaluator.objective(beta, gamma, knots)
            # constraints as (G, dG/dgamma, dG/daknots)
            cons = [(G, dG, None) for G, dG in volume_constraints(gamma, s)]
            if s.omega_max is not None:
                _, om = evaluator.angles()
                G3, dG3 = angular_speed_bound(om, s.omega_max, s.p_G3)
                cons.append((G3, None, evaluator.angles_T(np.zeros_like(dG3), dG3)))
            if mu is None:
                mu = np.zeros(len(cons))
            hist.beta.append(beta)
            hist.J.append(J)
            hist.G.append([c[0] for c in cons])
            if callback is not None:
                callback(beta, J, cons)
            if (J_prev is not None and abs(J - J_prev) <= s.tol * abs(J_prev)
                    and all(c[0] <= 0.0 for c in cons)):
                stopped = True
                break
            grads = evaluator.gradient()
            dg, dk = grads[0], grads[1]
            d_g = _unit(sign * np.asarray(dg))
            d_a = _unit(sign * np.asarray(grads[2])) if rot else None
            for j, (G, dGg, dGa) in enumerate(cons):
                wgt = max(0.0, s.rho * G + mu[j])
                if dGg is not None:
                    d_g = d_g - wgt * _unit(dGg)
                if dGa is not None:
                    d_a = d_a - wgt * _unit(dGa)
            d_g = _unit(d_g)
            d_k = _unit(sign * np.asarray(dk))
            if rot:
                d_a = _unit(d_a)
            if prev_g is not None:
                lim_g = _adapt(lim_g, d_g, prev_g, s.gamma_step)
                lim_k = _adapt(lim_k, d_k, prev_k, s.pos_step)
                if rot:
                    lim_a = _adapt(lim_a, d_a, prev_a, s.ang_step)
            prev_g, prev_k, prev_a = d_g, d_k, d_a
            gamma = np.clip(gamma + lim_g * d_g, 0.0, 1.0)
            knots = np.clip(knots + lim_k * d_k, -s.pos_bound, s.pos_bound)
            if rot:
                aknots = np.clip(aknots + lim_a * d_a, -s.ang_bound, s.ang_bound)
            for j, (G, _, _) in enumerate(cons):
                mu[j] = max(0.0, mu[j] + s.rho * G)
            J_prev = J
        hist.stopped_early.append(stopped)
    if rot:
        return gamma, knots, aknots, hist
    return gamma, knots, hist


class SolverEvaluator:
    """Forward and adjoint solves through the CUDA library for ``run``: one context per beta, created on first use.
    With periodic=True (Sec. 3.3) the final state of each forward solve is the initial state of the next, and the
    adjoint state at n = 0 of each reverse sweep is added to the terminal adjoint state of the next, across betas
    too."""

    def __init__(self, workload: dict, periodic: bool = False):
        self.w = workload
        self.periodic = periodic
        self.solvers = {}
        self.state = None
        self.lam0 = None
        self.current = None

    def objective(self, beta, gamma, knots, aknots=None):
        from .binding import Solver

        if beta not in self.solvers:
            self.solvers[beta] = Solver.from_workload(dict(self.w, beta=float(beta)))
        s = self.solvers[beta]
        if self.periodic and self.state is not None:
            s.set_initial_state(*self.state)
        if self.periodic and self.lam0 is not None:
            s.set_adjoint_terminal(*self.lam0)
        J = s.forward(gamma, knots, aknots=aknots)
        if self.periodic:
            self.state = s.state()
        self.current = s
        return J

    def gradient(self):
        g = self.current.adjoint()
        if self.periodic:
            self.lam0 = self.current.adjoint_initial()
        if self.current.params.K_w > 0:
            return g[0], g[1], self.current.angle_gradient()
        return g

    def angles(self):
        return self.current.angles()

    def angles_T(self, g_theta, g_omega):
        return self.current.angles_T(g_theta, g_omega)

    def close(self):
        for s in self.solvers.values():
            s.close()
        self.solvers = {}
