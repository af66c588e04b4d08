"""A rigidly rotating body on the CUDA path against the FP64 oracle (Sec. 2.3 Eqs. rigid_body_position,
rigid_body_velocity, kappa, u_s with theta != 0; Sec. 2.4 Eqs. psi_filtered, theta, omega; Sec. 2.5 Eq. dJdpsi).

The oracle maps the rotated design lattice with a dense weight matrix (map_rotated) and differentiates it exactly;
the CUDA path gathers from the rotated candidates per footprint-box node, differentiates the same sums, and applies
the transposed mapping on the design side.  Cases: both lattices, both transfer kernels, both precisions, the
checkpointed reverse sweeps, the gradient modes, theta = 0 against the translation path, and a body across the
periodic seam.
"""
import numpy as np
import pytest

from helpers import oracle_run_rot, rel_l2, rel_max, tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10, 1e-10), "fp32": (1e-5, 1e-4, 1e-3)}
ROT = dict(K_w=5, R_w=8.0)
# probe boxes at the body's downstream edge, so that J is not rounding-dominated over the short horizons
PROBE = {"D2Q9": dict(probe_lo=(38, 10), probe_hi=(48, 27)), "D3Q15": dict(probe_lo=(22, 4, 3), probe_hi=(28, 14, 10))}


def rot_workload(lattice, **over):
    return tiny_workload(lattice, **dict(PROBE[lattice], **ROT, **over))


def angle_knots(w, base=0.6, amp=0.03, seed=21):
    # a large angle (the rotated lattice far from the analysis axes) with a slow variation: the rim of the design grid
    # (arms up to about 11 cells) moves at most about 0.1 cell per step, within the stability limit
    rng = np.random.default_rng(seed)
    return base + rng.uniform(-amp, amp, w["K_w"])


def gpu_rot(w, gamma, knots, aknots):
    s = Solver.from_workload(w)
    J = s.forward(gamma, knots, aknots=aknots)
    p, u = s.state()
    dg, dk = s.adjoint()
    da = s.angle_gradient()
    gth, gom = s.step_angle_sensitivities()
    st = s.stats()
    s.close()
    return dict(J=J, p=p, u=u, dgamma=dg, dknots=dk, daknots=da, gth=gth, gom=gom, stats=st)


def check(w, aknots=None, ref=None):
    tf, tu, tg = TOL[w["precision"]]
    gamma, knots = draw_gamma(w), draw_knots(w)
    aknots = angle_knots(w) if aknots is None else aknots
    g = gpu_rot(w, gamma, knots, aknots)
    o = ref if ref is not None else oracle_run_rot(w, gamma, knots, aknots)
    assert abs(g["J"] - o["J"]) <= tf * abs(o["J"]), (g["J"], o["J"])
    assert rel_max(g["p"], o["p"]) <= tf
    assert rel_max(g["u"], o["u"]) <= tu
    mode = w.get("mode", "joint")
    if mode != "motion":
        assert rel_l2(g["dgamma"], o["dgamma"]) <= tg
    if mode != "shape":
        assert rel_l2(g["dknots"], o["dknots"]) <= tg
        assert rel_l2(g["daknots"], o["daknots"]) <= tg
        assert rel_l2(g["gth"][1:], o["gth"][1:]) <= tg and rel_l2(g["gom"][1:], o["gom"][1:]) <= tg
    else:
        assert np.all(g["daknots"] == 0)
    return g, o


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q15"])
@pytest.mark.parametrize("kernel", ["linear", "cosine"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rotating_body_matches_oracle(lattice, kernel, prec):
    nt = 24 if lattice == "D2Q9" else 12
    w = rot_workload(lattice, kernel=kernel, precision=prec, Nt=nt)
    g, o = check(w)
    assert np.abs(o["daknots"]).max() > 0 and np.abs(o["gom"]).max() > 0


@pytest.mark.parametrize("ckpt,rows", [("sqrt", 1), ("revolve", 8), ("revolve", 1)])
def test_rotating_body_checkpointed(ckpt, rows):
    w = rot_workload("D3Q15", precision="fp64", Nt=13, ckpt=ckpt, ckpt_slots=2, seg_len=4, tile_rows=1,
                     tile_rows_adj=rows)
    g, _ = check(w)
    assert g["stats"]["recompute_steps"] > 0


@pytest.mark.parametrize("mode", ["shape", "motion"])
def test_rotating_body_gradient_modes(mode):
    check(rot_workload("D2Q9", precision="fp64", Nt=20, mode=mode))


def test_zero_angle_equals_translation():
    # theta = 0 at every step: the rotated gather reproduces the translation path
    w = tiny_workload("D2Q9", precision="fp64", Nt=30, **PROBE["D2Q9"])
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    J0 = s.forward(gamma, knots)
    dg0, dk0 = s.adjoint()
    s.close()
    g = gpu_rot(dict(w, **ROT), gamma, knots, np.zeros(ROT["K_w"]))
    assert abs(g["J"] - J0) <= 1e-12 * abs(J0)
    assert rel_l2(g["dgamma"], dg0) <= 1e-12 and rel_l2(g["dknots"], dk0) <= 1e-12


OAR_ROT = dict(objective="J2", w_D=0.3, drag_span=9.0, w_T=0.7, l_m=5.0)


@pytest.mark.parametrize("lattice,kernel,prec", [("D2Q9", "linear", "fp64"), ("D2Q9", "cosine", "fp64"),
                                                 ("D3Q15", "linear", "fp64"), ("D2Q9", "linear", "fp32"),
                                                 ("D3Q15", "linear", "fp32")])
def test_rotating_oar_matches_oracle(lattice, kernel, prec):
    # objective J2 with the torque term (Eq. objective2): force, drag work and torque work on the design grid of a
    # rotating body, and their adjoint source and explicit derivatives (kappa^ref, position, u^G, theta, omega)
    nt = 24 if lattice == "D2Q9" else 12
    w = rot_workload(lattice, kernel=kernel, precision=prec, Nt=nt, **OAR_ROT)
    g, o = check(w)
    assert abs(o["J"]) > 0 and np.abs(o["daknots"]).max() > 0


@pytest.mark.parametrize("ckpt", ["sqrt", "revolve"])
def test_rotating_oar_checkpointed(ckpt):
    w = rot_workload("D2Q9", precision="fp64", Nt=21, ckpt=ckpt, ckpt_slots=2, seg_len=4, **OAR_ROT)
    g, _ = check(w)
    assert g["stats"]["recompute_steps"] > 0


def test_rotating_oar_torque_term_counts():
    # the same run with and without the torque weight: the torque term's share is visible in J
    w0 = rot_workload("D2Q9", precision="fp64", Nt=20, **dict(OAR_ROT, w_T=0.0))
    w1 = rot_workload("D2Q9", precision="fp64", Nt=20, **OAR_ROT)
    g0, _ = check(w0)
    g1, _ = check(w1)
    assert abs(g1["J"] - g0["J"]) > 1e-6 * abs(g0["J"])


def test_rotating_body_across_periodic_seam():
    w = rot_workload("D2Q9", precision="fp64", Nt=20, base_center=(3.0, 18.0), probe_lo=(8, 10), probe_hi=(18, 27))
    check(w)
