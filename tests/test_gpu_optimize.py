"""The projected-gradient step and the optimisation driver (the 256x128x128 workload's device iterations)."""
import numpy as np
import pytest

from helpers import tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.optimize import gradient_step_dev, optimize
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu


def test_gradient_step_matches_numpy():
    import torch

    rng = np.random.default_rng(3)
    for n in (1, 1000, 300001):
        g, x = rng.standard_normal(n), rng.uniform(0.0, 1.0, n)
        d_g, d_x = torch.tensor(g, device="cuda"), torch.tensor(x, device="cuda")
        gradient_step_dev(d_g, d_x, 0.05, 0.0, 1.0)
        ref = np.clip(x + 0.05 * g / np.max(np.abs(g)), 0.0, 1.0)
        assert np.max(np.abs(d_x.cpu().numpy() - ref)) <= 1e-15
    d_x = torch.tensor(x, device="cuda")
    gradient_step_dev(torch.zeros_like(d_x), d_x, 0.05, 0.0, 1.0)  # zero gradient: unchanged
    assert np.array_equal(d_x.cpu().numpy(), x)


def test_optimize_increases_J():
    w = tiny_workload("D2Q9", precision="fp64", Nt=40)
    s = Solver.from_workload(w)
    gamma, knots, hist = optimize(s, draw_gamma(w), draw_knots(w), iters=5, gamma_step=0.05, pos_step=0.5,
                                  pos_bound=w["amp"])
    assert len(hist) == 5 and hist[-1] > hist[0]
    assert np.all((gamma >= 0.0) & (gamma <= 1.0)) and np.all(np.abs(knots) <= w["amp"])
    s.close()


def test_algorithm1_on_the_cuda_solver_with_periodic_warm_start():
    # beta continuation over two values with the solid-volume constraint, each forward started from the previous
    # one's final state (Sec. 3.3); J and the gradients come from the CUDA library
    from paper_2608_01071_b300.algorithm1 import Settings, SolverEvaluator, run

    w = tiny_workload("D2Q9", precision="fp64", Nt=30)
    ev = SolverEvaluator(w, periodic=True)
    s = Settings(betas=(1.0, 4.0), n_opt=3, gamma_step=0.05, pos_step=0.3, pos_bound=w["amp"], V_max_solid=0.7,
                 tol=0.0)
    gamma, knots, h = run(ev, np.clip(draw_gamma(w), 0.0, 0.6), draw_knots(w), s)
    ev.close()
    assert h.beta == [1.0] * 3 + [4.0] * 3 and all(np.isfinite(h.J))
    assert len(ev.solvers) == 0 and np.all((gamma >= 0.0) & (gamma <= 1.0))
    # the warm start changes the forward: the second J of beta 1 differs from a cold start at the same design
    assert h.J[1] != h.J[0]


def test_angular_speed_constraint_from_the_library():
    # G3 (Eq. constraint3) from the library's omega_n and its chain to the angle knots, against the oracle's
    # angles and angle_gradient; then a few iterations of the driver with angle knots on the CUDA solver
    import oracle as O
    from helpers import oracle_problem, rel_l2, tiny_workload
    from paper_2608_01071_b300.algorithm1 import Settings, SolverEvaluator, angular_speed_bound, run

    w = tiny_workload("D2Q9", precision="fp64", Nt=24, K_w=5, R_w=8.0, probe_lo=(38, 10), probe_hi=(48, 27))
    gamma, knots = draw_gamma(w), draw_knots(w)
    aknots = 0.3 + np.random.default_rng(3).uniform(-0.03, 0.03, 5)
    ev = SolverEvaluator(w)
    ev.objective(1.0, gamma, knots, aknots)
    th, om = ev.angles()
    P = oracle_problem(w)
    tho, omo = O.angles(aknots, P.Nt, P.R_w)
    assert np.max(np.abs(th - tho)) <= 1e-13 and np.max(np.abs(om - omo)) <= 1e-13
    G3, g = angular_speed_bound(om, 0.002, 8.0)
    G3o, go = O.angular_speed_bound(omo, 0.002, 8.0)
    assert abs(G3 - G3o) <= 1e-12 * abs(G3o)
    da = ev.angles_T(np.zeros_like(g), g)
    dao = O.angle_gradient(P, np.zeros_like(go), go, 5)
    assert rel_l2(da, dao) <= 1e-12
    ev.close()
    s = Settings(betas=(1.0,), n_opt=4, omega_max=0.002, p_G3=8.0, ang_step=0.005, gamma_step=0.05, pos_step=0.2,
                 pos_bound=2.0, tol=0.0)
    ev = SolverEvaluator(w)
    _, _, a, h = run(ev, gamma, knots, s, aknots=aknots)
    ev.close()
    assert len(h.J) == 4 and all(np.isfinite(h.J)) and len(h.G[0]) == 1
