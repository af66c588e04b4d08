"""Python binding of the C ABI: one ``Solver`` per library context.  Argument marshalling only.

Host arrays use the math index order [x, y(, z)]; they are passed to the library in its flat x-fastest
order (``a.T`` in C order) and converted back on return.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _abi

_MAP = {"linear": _abi.LKS_MAP_LINEAR, "cosine": _abi.LKS_MAP_COSINE}
_PREC = {"fp64": _abi.LKS_FP64, "fp32": _abi.LKS_FP32}
_CKPT = {"full": _abi.LKS_CKPT_FULL, "sqrt": _abi.LKS_CKPT_SQRT, "revolve": _abi.LKS_CKPT_REVOLVE}
_MODE = {"joint": _abi.LKS_MODE_JOINT, "shape": _abi.LKS_MODE_SHAPE, "motion": _abi.LKS_MODE_MOTION}
_OBJ = {"J1": _abi.LKS_OBJ_FLOW, "J2": _abi.LKS_OBJ_OAR}


class LKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def params_from_workload(w: dict) -> _abi.lks_params:
    """Fill an lks_params from a workload description (plain data; see ``workloads``)."""
    lib = _abi.load()
    p = _abi.lks_params()
    lib.lks_default_params(C.byref(p))
    d = len(w["shape"])
    p.lattice = _abi.LKS_D2Q9 if w["lattice"] == "D2Q9" else _abi.LKS_D3Q15
    for a in range(3):
        p.n[a] = w["shape"][a] if a < d else 1
        p.periodic[a] = int(bool(w["periodic"][a])) if a < d else 1
        p.nd[a] = w["design"][a] if a < d else 1
        p.probe_lo[a] = w["probe_lo"][a] if a < d else 0
        p.probe_hi[a] = w["probe_hi"][a] if a < d else 1
        p.direction[a] = w["direction"][a] if a < d else 0.0
        bc = w.get("base_center")
        p.base_center[a] = bc[a] if (bc is not None and a < d) else math.nan
    for (axis, side), vel in w.get("wall_velocity", {}).items():
        for b in range(d):
            p.wall_velocity[axis][side][b] = vel[b]
    p.nu = w["nu"]
    p.kappa_max = w["kappa_max"]
    p.q = w["q"]
    p.margin = w["margin"]
    p.map_kernel = _MAP[w["kernel"]]
    p.Nt = w["Nt"]
    p.K = w["K"]
    p.R_t = w["R_t"]
    p.filter_R = w["filter_R"]
    p.beta = w["beta"]
    p.eta = w["eta"]
    p.precision = _PREC[w["precision"]]
    p.ckpt = _CKPT[w["ckpt"]]
    p.ckpt_slots = w.get("ckpt_slots", 0)
    p.seg_len = w.get("seg_len", 0)
    p.ckpt_bytes = int(w.get("ckpt_bytes", 0))
    p.mode = _MODE[w.get("mode", "joint")]
    p.u_crit = w.get("u_crit", 0.3)
    p.tile_rows = w.get("tile_rows", 0)
    p.tile_rows_adj = w.get("tile_rows_adj", 0)
    p.tile_rows_rec = w.get("tile_rows_rec", 0)
    p.phi_var = w.get("phi_var", 0.0)
    objective = w.get("objective", "J1")
    if objective not in _OBJ:
        raise ValueError(f"objective must be one of {sorted(_OBJ)}, not {objective!r}")
    p.objective = _OBJ[objective]
    p.w_D = w.get("w_D", 0.0)
    p.drag_span = w.get("drag_span", 1.0)
    p.w_T = w.get("w_T", 0.0)
    p.l_m = w.get("l_m", 1.0)
    p.K_w = w.get("K_w", 0)
    adj = w.get("adjoint", "discrete")
    if adj not in ("discrete", "alks"):
        raise ValueError(f"adjoint must be 'discrete' or 'alks', not {adj!r}")
    p.adjoint = 1 if adj == "alks" else 0
    p.R_w = w.get("R_w", 1.0)
    return p


def _flat(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Solver:
    """One library context (device state owned by the library)."""

    def __init__(self, params: _abi.lks_params):
        self.lib = _abi.load()
        self.params = params
        self.d = 2 if params.lattice == _abi.LKS_D2Q9 else 3
        self.shape = tuple(params.n[a] for a in range(self.d))
        self.design = tuple(params.nd[a] for a in range(self.d))
        self.K = params.K
        self.Nt = params.Nt
        h = C.c_void_p()
        rc = self.lib.lks_create(C.byref(params), C.byref(h))
        if rc != 0:
            raise LKSError(rc, self.lib.lks_last_error_string(None).decode())
        self.h = h

    @classmethod
    def from_workload(cls, w: dict) -> "Solver":
        return cls(params_from_workload(w))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise LKSError(rc, self.lib.lks_last_error_string(self.h).decode())

    # host-pointer calls -------------------------------------------------------------------------
    def set_angle_knots(self, aknots):
        """Angle knots (radians, K_w values) of the rotating body for the following forwards."""
        a = np.ascontiguousarray(aknots, dtype=np.float64)
        self._check(self.lib.lks_set_angle_knots(self.h, _dptr(a)))

    def angle_gradient(self):
        """dJ/d(angle knots) of the last adjoint."""
        out = np.zeros(self.params.K_w)
        self._check(self.lib.lks_get_angle_gradient(self.h, _dptr(out)))
        return out

    def angles(self):
        """(theta_n, omega_n), n = 0..Nt, of the last forward."""
        th = np.zeros(self.Nt + 1)
        om = np.zeros(self.Nt + 1)
        self._check(self.lib.lks_get_angles(self.h, _dptr(th), _dptr(om)))
        return th, om

    def angles_T(self, g_theta, g_omega):
        """Per-step sensitivities (g_theta, g_omega) -> gradient with respect to the angle knots."""
        gt = np.ascontiguousarray(g_theta, dtype=np.float64)
        go = np.ascontiguousarray(g_omega, dtype=np.float64)
        out = np.zeros(self.params.K_w)
        self._check(self.lib.lks_angles_T(self.h, _dptr(gt), _dptr(go), _dptr(out)))
        return out

    def step_angle_sensitivities(self):
        gth = np.zeros(self.Nt + 1)
        gom = np.zeros(self.Nt + 1)
        self._check(self.lib.lks_get_step_angle_sensitivities(self.h, _dptr(gth), _dptr(gom)))
        return gth, gom

    def forward(self, gamma, knots, aknots=None) -> float:
        if aknots is not None:
            self.set_angle_knots(aknots)
        g = _flat(gamma)
        k = np.ascontiguousarray(knots, dtype=np.float64)
        J = C.c_double()
        self._check(self.lib.lks_forward(self.h, _dptr(g), _dptr(k), C.byref(J)))
        return J.value

    def adjoint(self):
        dg = np.zeros(self.design[::-1])
        dk = np.zeros((self.K, self.d))
        self._check(self.lib.lks_adjoint(self.h, _dptr(dg), _dptr(dk)))
        return dg.T.copy(), dk

    def state(self):
        N = int(np.prod(self.shape))
        p = np.zeros(N)
        u = np.zeros(self.d * N)
        self._check(self.lib.lks_get_state(self.h, _dptr(p), _dptr(u)))
        p = p.reshape(self.shape[::-1]).T.copy()
        u = np.stack([u[a * N:(a + 1) * N].reshape(self.shape[::-1]).T for a in range(self.d)])
        return p, u

    def set_initial_state(self, p=None, u=None):
        """Initial state of the following forwards (arrays as returned by state()); None restores the default."""
        if p is None and u is None:
            self._check(self.lib.lks_set_initial_state(self.h, None, None))
            return
        pf = np.ascontiguousarray(np.asarray(p, dtype=np.float64).T).ravel()
        uf = np.concatenate([np.ascontiguousarray(np.asarray(u[a], dtype=np.float64).T).ravel() for a in range(self.d)])
        self._check(self.lib.lks_set_initial_state(self.h, _dptr(pf), _dptr(uf)))

    def set_adjoint_terminal(self, lam_p=None, lam_u=None):
        """Terminal adjoint state added before the following reverse sweeps (arrays as returned by
        adjoint_initial()); None removes it."""
        if lam_p is None and lam_u is None:
            self._check(self.lib.lks_set_adjoint_terminal(self.h, None, None))
            return
        pf = np.ascontiguousarray(np.asarray(lam_p, dtype=np.float64).T).ravel()
        uf = np.concatenate([np.ascontiguousarray(np.asarray(lam_u[a], dtype=np.float64).T).ravel() for a in range(self.d)])
        self._check(self.lib.lks_set_adjoint_terminal(self.h, _dptr(pf), _dptr(uf)))

    def adjoint_initial(self):
        """lambda_0 = dJ/d(p_0, u_0) of the last adjoint, as (lam_p, lam_u) in the layout of state()."""
        N = int(np.prod(self.shape))
        p = np.zeros(N)
        u = np.zeros(self.d * N)
        self._check(self.lib.lks_get_adjoint_initial(self.h, _dptr(p), _dptr(u)))
        p = p.reshape(self.shape[::-1]).T.copy()
        u = np.stack([u[a * N:(a + 1) * N].reshape(self.shape[::-1]).T for a in range(self.d)])
        return p, u

    def step_sensitivities(self):
        gs = np.zeros((self.Nt + 1, self.d))
        gu = np.zeros((self.Nt + 1, self.d))
        self._check(self.lib.lks_get_step_sensitivities(self.h, _dptr(gs), _dptr(gu)))
        return gs, gu

    def objective_terms(self):
        """(E, V) of the last forward: mean and variance of n.u over O_target and the horizon (J = E - phi_var V)."""
        E, V = C.c_double(), C.c_double()
        self._check(self.lib.lks_get_objective_terms(self.h, C.byref(E), C.byref(V)))
        return E.value, V.value

    def status(self):
        """Waits for the last forward; raises LKSError (LKS_EUNSTABLE) if it was unstable."""
        self._check(self.lib.lks_get_status(self.h))

    def set_timing(self, on: bool):
        self._check(self.lib.lks_set_timing(self.h, 1 if on else 0))

    def set_graphs(self, on: bool):
        self._check(self.lib.lks_set_graphs(self.h, 1 if on else 0))

    def stats(self) -> dict:
        s = _abi.lks_stats()
        self._check(self.lib.lks_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    # device-pointer calls (torch tensors: contiguous float64 on the current device, flat x-fastest) ---
    def forward_dev(self, d_gamma, d_knots, d_J, stream=None):
        self._check(self.lib.lks_forward_dev(self.h, C.c_void_p(d_gamma.data_ptr()), C.c_void_p(d_knots.data_ptr()),
                                             C.c_void_p(d_J.data_ptr()), _stream_ptr(stream)))

    def adjoint_dev(self, d_dgamma, d_dknots, stream=None):
        self._check(self.lib.lks_adjoint_dev(self.h, C.c_void_p(d_dgamma.data_ptr()) if d_dgamma is not None else None,
                                             C.c_void_p(d_dknots.data_ptr()) if d_dknots is not None else None,
                                             _stream_ptr(stream)))

    def density_filter_dev(self, d_in, d_out, transpose=False, stream=None):
        f = self.lib.lks_density_filter_T_dev if transpose else self.lib.lks_density_filter_dev
        self._check(f(self.h, C.c_void_p(d_in.data_ptr()), C.c_void_p(d_out.data_ptr()), _stream_ptr(stream)))

    def motion_filter_dev(self, d_in, d_out, transpose=False, stream=None):
        f = self.lib.lks_motion_filter_T_dev if transpose else self.lib.lks_motion_filter_dev
        self._check(f(self.h, C.c_void_p(d_in.data_ptr()), C.c_void_p(d_out.data_ptr()), _stream_ptr(stream)))

    def interp_positions_dev(self, d_filt, d_s, d_uG, stream=None):
        self._check(self.lib.lks_interp_positions_dev(self.h, C.c_void_p(d_filt.data_ptr()), C.c_void_p(d_s.data_ptr()),
                                                      C.c_void_p(d_uG.data_ptr()), _stream_ptr(stream)))

    def interp_positions_T_dev(self, d_gs, d_guG, d_out, stream=None):
        self._check(self.lib.lks_interp_positions_T_dev(self.h, C.c_void_p(d_gs.data_ptr()), C.c_void_p(d_guG.data_ptr()),
                                                        C.c_void_p(d_out.data_ptr()), _stream_ptr(stream)))


    # host-array calls (numpy float64; design arrays flat x-fastest, knots and positions row-major) ---------
    def _ptr(self, a):
        return a.ctypes.data_as(C.POINTER(C.c_double))

    def density_filter(self, x, transpose=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(x)
        f = self.lib.lks_density_filter_T if transpose else self.lib.lks_density_filter
        self._check(f(self.h, self._ptr(x), self._ptr(out)))
        return out

    def motion_filter(self, x, transpose=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(x)
        f = self.lib.lks_motion_filter_T if transpose else self.lib.lks_motion_filter
        self._check(f(self.h, self._ptr(x), self._ptr(out)))
        return out

    def interp_positions(self, filtered, Nt):
        filtered = np.ascontiguousarray(filtered, dtype=np.float64)
        s = np.empty((Nt + 1, filtered.shape[1]))
        uG = np.empty_like(s)
        self._check(self.lib.lks_interp_positions(self.h, self._ptr(filtered), self._ptr(s), self._ptr(uG)))
        return s, uG

    def interp_positions_T(self, gs, guG, K):
        gs = np.ascontiguousarray(gs, dtype=np.float64)
        guG = np.ascontiguousarray(guG, dtype=np.float64)
        out = np.empty((K, gs.shape[1]))
        self._check(self.lib.lks_interp_positions_T(self.h, self._ptr(gs), self._ptr(guG), self._ptr(out)))
        return out


def projection(x, beta, eta):
    """Heaviside projection and its derivative of a host array (through the library's kernel)."""
    lib = _abi.load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    out, dout = np.empty_like(x), np.empty_like(x)
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = lib.lks_projection(x.size, beta, eta, p(x), p(out), p(dout))
    if rc != 0:
        raise LKSError(rc, lib.lks_strerror(rc).decode())
    return out, dout


def projection_dev(d_in, d_out, d_dout, beta, eta, stream=None):
    lib = _abi.load()
    rc = lib.lks_projection_dev(d_in.numel(), beta, eta, C.c_void_p(d_in.data_ptr()),
                                C.c_void_p(d_out.data_ptr()) if d_out is not None else None,
                                C.c_void_p(d_dout.data_ptr()) if d_dout is not None else None, _stream_ptr(stream))
    if rc != 0:
        raise LKSError(rc, lib.lks_strerror(rc).decode())


class Batch:
    """A batched parameter study (one library batch; every instance has its own context)."""

    def __init__(self, workloads):
        self.lib = _abi.load()
        self.params = (_abi.lks_params * len(workloads))(*[params_from_workload(w) for w in workloads])
        self.count = len(workloads)
        h = C.c_void_p()
        rc = self.lib.lks_batch_create(self.count, self.params, C.byref(h))
        if rc != 0:
            raise LKSError(rc, self.lib.lks_batch_last_error(None).decode())
        self.h = h
        self.d = [2 if p.lattice == _abi.LKS_D2Q9 else 3 for p in self.params]
        self.K = [p.K for p in self.params]
        self.design = [tuple(p.nd[a] for a in range(dd)) for p, dd in zip(self.params, self.d)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.lks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise LKSError(rc, self.lib.lks_batch_last_error(self.h).decode())

    def context_stats(self, i) -> dict:
        s = _abi.lks_stats()
        rc = self.lib.lks_get_stats(self.lib.lks_batch_context(self.h, i), C.byref(s))
        self._check(rc)
        return {f: getattr(s, f) for f, _ in s._fields_}

    def forward_dev(self, d_gammas, d_knots, d_J, stream=None):
        ga = (C.c_void_p * self.count)(*[t.data_ptr() for t in d_gammas])
        ka = (C.c_void_p * self.count)(*[t.data_ptr() for t in d_knots])
        self._check(self.lib.lks_batch_forward_dev(self.h, ga, ka, C.c_void_p(d_J.data_ptr()), _stream_ptr(stream)))

    def adjoint_dev(self, d_dgammas, d_dknots, stream=None):
        ga = (C.c_void_p * self.count)(*[t.data_ptr() for t in d_dgammas])
        ka = (C.c_void_p * self.count)(*[t.data_ptr() for t in d_dknots])
        self._check(self.lib.lks_batch_adjoint_dev(self.h, ga, ka, _stream_ptr(stream)))
