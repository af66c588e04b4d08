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
