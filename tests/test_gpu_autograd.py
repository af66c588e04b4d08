"""torch.autograd.Function over the CUDA forward/adjoint, against the FP64 oracle."""
import pytest

from helpers import oracle_run, rel_l2, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
def test_autograd_matches_oracle(lattice):
    import torch

    from paper_2608_01071_b300.autograd import LKSFunction

    w = tiny_workload(lattice, precision="fp32", ckpt="sqrt")
    gamma, knots = draw_gamma(w), draw_knots(w)
    o = oracle_run(w, gamma, knots)
    s = Solver.from_workload(w)
    g = torch.tensor(gamma, device="cuda", requires_grad=True)
    k = torch.tensor(knots, device="cuda", requires_grad=True)
    J = LKSFunction.apply(g, k, s)
    (2.5 * J).backward()
    assert abs(J.item() - o["J"]) <= 1e-5 * abs(o["J"])
    assert rel_l2(g.grad.cpu().numpy(), 2.5 * o["dgamma"]) <= 1e-3
    assert rel_l2(k.grad.cpu().numpy(), 2.5 * o["dknots"]) <= 1e-3
    # a second pass on the same solver (graph replay) with new inputs
    g2 = torch.tensor(gamma * 0.8, device="cuda", requires_grad=True)
    J2 = LKSFunction.apply(g2, k.detach(), s)
    J2.backward()
    o2 = oracle_run(w, gamma * 0.8, knots)
    assert rel_l2(g2.grad.cpu().numpy(), o2["dgamma"]) <= 1e-3
    s.close()
