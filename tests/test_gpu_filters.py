"""The filter calls of the C ABI (design density filter and its transpose, Heaviside projection, temporal motion
filter and its transpose, position interpolation and its transpose), host-pointer and device-pointer variants,
against the FP64 oracle's functions of Eqs. filtering, projection, chi_filtered and u_g."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_problem, rel_max, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.binding import projection, projection_dev

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
def test_filter_calls_match_oracle(lattice):
    import torch

    w = tiny_workload(lattice, precision="fp64")
    P = oracle_problem(w)
    rng = np.random.default_rng(5)
    s = Solver.from_workload(w)
    dev = torch.device("cuda", 0)
    flat = lambda a: np.ascontiguousarray(a.T).ravel()  # design arrays: x fastest in the C ABI

    # density filter and transpose
    gamma = rng.uniform(0.0, 1.0, tuple(w["design"]))
    g = rng.normal(size=tuple(w["design"]))
    ref_f, ref_t = O.density_filter(gamma, P.filter_R), O.density_filter_T(g, P.filter_R)
    assert rel_max(s.density_filter(flat(gamma)), flat(ref_f)) <= TOL
    assert rel_max(s.density_filter(flat(g), transpose=True), flat(ref_t)) <= TOL
    d_in = torch.tensor(flat(gamma), device=dev)
    d_out = torch.empty_like(d_in)
    s.density_filter_dev(d_in, d_out)
    torch.cuda.synchronize()
    assert rel_max(d_out.cpu().numpy(), flat(ref_f)) <= TOL

    # projection and its derivative
    x = rng.uniform(0.0, 1.0, 1000)
    out, dout = projection(x, 6.0, 0.4)
    assert rel_max(out, O.projection(x, 6.0, 0.4)) <= TOL
    assert rel_max(dout, O.projection_deriv(x, 6.0, 0.4)) <= TOL
    d_x = torch.tensor(x, device=dev)
    d_o, d_do = torch.empty_like(d_x), torch.empty_like(d_x)
    projection_dev(d_x, d_o, d_do, 6.0, 0.4)
    torch.cuda.synchronize()
    assert rel_max(d_o.cpu().numpy(), O.projection(x, 6.0, 0.4)) <= TOL

    # temporal motion filter and transpose (knots K x d, row-major)
    D = len(w["shape"])
    knots = rng.normal(size=(P.K, D))
    filt = s.motion_filter(knots)
    assert rel_max(filt, O.motion_filter(knots, P.Nt, P.R_t)) <= TOL
    gk = rng.normal(size=(P.K, D))
    assert rel_max(s.motion_filter(gk, transpose=True), O.motion_filter_T(gk, P.Nt, P.R_t)) <= TOL

    # interpolation to every step, u^G as the backward difference (u^G_0 = u^G_1), and the transpose
    sp, uG = s.interp_positions(filt, P.Nt)
    ref_s = O.interp_matrix(P.K, P.Nt) @ filt
    ref_u = np.zeros_like(ref_s)
    ref_u[1:] = ref_s[1:] - ref_s[:-1]
    ref_u[0] = ref_u[1]
    assert rel_max(sp, ref_s) <= TOL and rel_max(uG, ref_u) <= TOL
    gs, gu = rng.normal(size=(P.Nt + 1, D)), rng.normal(size=(P.Nt + 1, D))
    gu[0] = 0.0  # u^G_0 enters no step
    ref_g = gs.copy()
    ref_g[1:] += gu[1:]
    ref_g[:-1] -= gu[1:]
    assert rel_max(s.interp_positions_T(gs, gu, P.K), O.interp_matrix(P.K, P.Nt).T @ ref_g) <= TOL
    s.close()
