"""Gradients of the CUDA path against central finite differences of its own objective.

- The 96x48 FP64 workload at its full size: 8 design cells drawn with seed 0 and 4 knots, h = 1e-6.
- The 512x256 workload's grid and design chain (filter, projection), in FP64 so that differences resolve, with
  the horizon cut to 60 steps: through the torch.autograd.Function, a directional central difference along a
  random direction in (gamma, knots) against the autograd gradient.
"""
import numpy as np
import pytest

from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots, workload

pytestmark = pytest.mark.gpu
H = 1e-6


def test_c1_central_differences():
    w = workload("d2q9_96x48_fp64")
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    s.forward(gamma, knots)
    dg, dk = s.adjoint()
    scale_g, scale_k = np.max(np.abs(dg)), np.max(np.abs(dk))
    rng = np.random.default_rng(0)
    cells = [(int(rng.integers(2, w["design"][0] - 2)), int(rng.integers(2, w["design"][1] - 2))) for _ in range(8)]
    for c in cells:
        e = np.zeros_like(gamma)
        e[c] = H
        fd = (s.forward(gamma + e, knots) - s.forward(gamma - e, knots)) / (2 * H)
        assert abs(fd - dg[c]) <= 1e-6 * scale_g, (c, fd, dg[c])
    for k in rng.choice(w["K"], 4, replace=False):
        e = np.zeros_like(knots)
        e[k, 0] = H
        fd = (s.forward(gamma, knots + e) - s.forward(gamma, knots - e)) / (2 * H)
        assert abs(fd - dk[k, 0]) <= 1e-6 * scale_k, (k, fd, dk[k, 0])
    s.close()


def test_c2_autograd_directional_difference():
    import torch

    from paper_2608_01071_b300.autograd import LKSFunction

    w = workload("d2q9_512x256_fp32", precision="fp64", Nt=60, K=6, R_t=15.0, amp=32.0 * 60 / 4000,
                 probe_lo=(300, 96), probe_hi=(340, 160))
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    g = torch.tensor(gamma, device="cuda", requires_grad=True)
    k = torch.tensor(knots, device="cuda", requires_grad=True)
    J = LKSFunction.apply(g, k, s)
    J.backward()
    rng = np.random.default_rng(1)
    vg, vk = rng.standard_normal(gamma.shape), rng.standard_normal(knots.shape)
    dd = float((g.grad.cpu().numpy() * vg).sum() + (k.grad.cpu().numpy() * vk).sum())
    with torch.no_grad():
        Jp = LKSFunction.apply(torch.tensor(gamma + H * vg, device="cuda"), torch.tensor(knots + H * vk, device="cuda"), s)
        Jm = LKSFunction.apply(torch.tensor(gamma - H * vg, device="cuda"), torch.tensor(knots - H * vk, device="cuda"), s)
    fd = (Jp.item() - Jm.item()) / (2 * H)
    assert abs(fd - dd) <= 1e-6 * abs(dd), (fd, dd)
    s.close()
