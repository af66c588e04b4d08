"""Test helpers: build the oracle's problem and the library's parameters from one workload description."""
import numpy as np

import oracle as O


def oracle_problem(w, **kw):
    d = len(w["shape"])
    P = O.Problem(lattice=w["lattice"], shape=tuple(w["shape"]), periodic=tuple(bool(v) for v in w["periodic"]),
                  nu=w["nu"], design=tuple(w["design"]), margin=w["margin"], kappa_max=w["kappa_max"], q=w["q"],
                  kernel=w["kernel"], Nt=w["Nt"], K=w["K"], R_t=w["R_t"], filter_R=w["filter_R"], beta=w["beta"],
                  eta=w["eta"], probe_lo=tuple(w["probe_lo"]), probe_hi=tuple(w["probe_hi"]),
                  direction=tuple(w["direction"]), base_center=w.get("base_center"),
                  wall_velocity=dict(w.get("wall_velocity", {})), phi_var=w.get("phi_var", 0.0),
                  objective=w.get("objective", "J1"), w_D=w.get("w_D", 0.0), drag_span=w.get("drag_span", 1.0),
                  w_T=w.get("w_T", 0.0), l_m=w.get("l_m", 1.0), R_w=w.get("R_w", 1.0))
    return P


def oracle_run(w, gamma, knots, state0=None, terminal=None):
    """J, dJ/dgamma, dJ/dknots, the final state (p, u) and lambda_0 from the oracle (state0: initial (p, u), or the
    default; terminal: (lam_p, lam_u) added to the terminal adjoint state)."""
    P = oracle_problem(w)
    kref, gt, gb = O.design_to_kref(P, gamma)
    s, uG = O.positions(knots, P.Nt, P.R_t)
    J, states = O.forward(P, kref, s, uG, store=True, state0=state0)
    lam0 = []
    g_kref, g_s, g_uG = O.adjoint(P, kref, s, uG, states, terminal=terminal, lambda0=lam0)
    g_kr = O.strip_margin(g_kref, P.margin)
    g_gb = g_kr * O.kappa_ref_deriv(gb, P.kappa_max, P.q)
    g_gt = g_gb * O.projection_deriv(gt, P.beta, P.eta)
    g_gamma = O.density_filter_T(g_gt, P.filter_R)
    g_knots = O.knot_gradient(P, g_s, g_uG)
    return dict(J=J, dgamma=g_gamma, dknots=g_knots, p=states[-1][0], u=states[-1][1], gs=g_s, guG=g_uG,
                lam0=lam0[0])


def rel_max(a, b):
    """max |a - b| / max |b| (field-relative error)."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def tiny_workload(lattice="D2Q9", **over):
    """A small workload spanning several tiles with ragged tails (for parity tests)."""
    if lattice == "D2Q9":
        w = dict(lattice="D2Q9", shape=(70, 37), periodic=(True, False), nu=0.03, design=(14, 11), margin=2,
                 kappa_max=2.0, q=0.1, kernel="linear", Nt=60, K=7, R_t=20.0, filter_R=1.6, beta=4.0, eta=0.5,
                 probe_lo=(50, 10), probe_hi=(62, 27), direction=(1.0, 0.0), precision="fp64", ckpt="full",
                 ckpt_slots=0, motion="sinusoids", amp=5.0, seed=11, wall_velocity={(1, 1): (0.02, 0.0)})
    else:
        w = dict(lattice="D3Q15", shape=(40, 19, 13), periodic=(True, False, False), nu=0.03, design=(8, 6, 5),
                 margin=2, kappa_max=2.0, q=0.1, kernel="linear", Nt=40, K=6, R_t=15.0, filter_R=1.5, beta=4.0,
                 eta=0.5, probe_lo=(30, 4, 3), probe_hi=(36, 14, 10), direction=(1.0, 0.0, 0.0), precision="fp64",
                 ckpt="full", ckpt_slots=0, motion="sinusoids", amp=2.5, seed=12)
    w.update(over)
    w.setdefault("name", "tiny")
    return w


def oracle_run_rot(w, gamma, knots, aknots):
    """The oracle with a rotating body (angle knots aknots): J, dJ/dgamma, dJ/dknots, dJ/daknots, the final state and
    the per-step dJ/dtheta_n, dJ/domega_n."""
    P = oracle_problem(w)
    kref, gt, gb = O.design_to_kref(P, gamma)
    s, uG = O.positions(knots, P.Nt, P.R_t)
    rot = O.angles(aknots, P.Nt, P.R_w)
    J, states = O.forward(P, kref, s, uG, store=True, rot=rot)
    g_kref, g_s, g_uG, g_th, g_om = O.adjoint(P, kref, s, uG, states, rot=rot)
    g_kr = O.strip_margin(g_kref, P.margin)
    g_gb = g_kr * O.kappa_ref_deriv(gb, P.kappa_max, P.q)
    g_gt = g_gb * O.projection_deriv(gt, P.beta, P.eta)
    return dict(J=J, dgamma=O.density_filter_T(g_gt, P.filter_R), dknots=O.knot_gradient(P, g_s, g_uG),
                daknots=O.angle_gradient(P, g_th, g_om, len(aknots)), p=states[-1][0], u=states[-1][1], gth=g_th,
                gom=g_om)
