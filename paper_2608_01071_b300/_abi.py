"""ctypes declarations of the C ABI in include/lks.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblks.so")

LKS_OK, LKS_EINVAL, LKS_ENOMEM, LKS_ECUDA, LKS_ESTATE, LKS_EUNSTABLE, LKS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LKS_D2Q9, LKS_D3Q15 = 9, 15
LKS_MAP_LINEAR, LKS_MAP_COSINE = 0, 1
LKS_FP64, LKS_FP32 = 0, 1
LKS_CKPT_FULL, LKS_CKPT_SQRT, LKS_CKPT_REVOLVE = 0, 1, 2
LKS_MODE_JOINT, LKS_MODE_SHAPE, LKS_MODE_MOTION = 0, 1, 2
LKS_OBJ_FLOW, LKS_OBJ_OAR = 0, 1
LKS_ADJ_DISCRETE, LKS_ADJ_ALKS = 0, 1


class lks_params(C.Structure):
    _fields_ = [
        ("size", C.c_uint32),
        ("lattice", C.c_int32),
        ("n", C.c_int32 * 3),
        ("periodic", C.c_int32 * 3),
        ("wall_velocity", ((C.c_double * 3) * 2) * 3),
        ("nu", C.c_double),
        ("kappa_max", C.c_double),
        ("q", C.c_double),
        ("nd", C.c_int32 * 3),
        ("margin", C.c_int32),
        ("map_kernel", C.c_int32),
        ("base_center", C.c_double * 3),
        ("probe_lo", C.c_int32 * 3),
        ("probe_hi", C.c_int32 * 3),
        ("direction", C.c_double * 3),
        ("Nt", C.c_int32),
        ("K", C.c_int32),
        ("R_t", C.c_double),
        ("filter_R", C.c_double),
        ("beta", C.c_double),
        ("eta", C.c_double),
        ("precision", C.c_int32),
        ("ckpt", C.c_int32),
        ("ckpt_slots", C.c_int32),
        ("seg_len", C.c_int32),
        ("ckpt_bytes", C.c_int64),
        ("mode", C.c_int32),
        ("u_crit", C.c_double),
        ("tile_rows", C.c_int32),
        ("tile_rows_adj", C.c_int32),
        ("tile_rows_rec", C.c_int32),
        ("phi_var", C.c_double),
        ("objective", C.c_int32),
        ("reserved_obj", C.c_int32),
        ("w_D", C.c_double),
        ("drag_span", C.c_double),
        ("K_w", C.c_int32),
        ("adjoint", C.c_int32),
        ("R_w", C.c_double),
        ("w_T", C.c_double),
        ("l_m", C.c_double),
    ]


class lks_stats(C.Structure):
    _fields_ = [
        ("forward_steps", C.c_int64),
        ("recompute_steps", C.c_int64),
        ("adjoint_steps", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("device_bytes", C.c_int64),
        ("ckpt_slots", C.c_int32),
        ("seg_len", C.c_int32),
        ("tile_rows_fwd", C.c_int32),
        ("tile_rows_adj", C.c_int32),
        ("tile_rows_rec", C.c_int32),
        ("pipelined", C.c_int32),
        ("ms_forward_steps", C.c_double),
        ("ms_recompute_steps", C.c_double),
        ("ms_adjoint_steps", C.c_double),
        ("ms_total", C.c_double),
    ]


_P = C.c_void_p
_D = C.POINTER(C.c_double)

# name -> (restype, argtypes)
PROTOTYPES = {
    "lks_default_params": (C.c_int, [C.POINTER(lks_params)]),
    "lks_create": (C.c_int, [C.POINTER(lks_params), C.POINTER(_P)]),
    "lks_destroy": (None, [_P]),
    "lks_last_error_string": (C.c_char_p, [_P]),
    "lks_strerror": (C.c_char_p, [C.c_int]),
    "lks_forward": (C.c_int, [_P, _D, _D, _D]),
    "lks_forward_dev": (C.c_int, [_P, _P, _P, _P, _P]),
    "lks_adjoint": (C.c_int, [_P, _D, _D]),
    "lks_adjoint_dev": (C.c_int, [_P, _P, _P, _P]),
    "lks_density_filter_dev": (C.c_int, [_P, _P, _P, _P]),
    "lks_density_filter_T_dev": (C.c_int, [_P, _P, _P, _P]),
    "lks_projection_dev": (C.c_int, [C.c_int64, C.c_double, C.c_double, _P, _P, _P, _P]),
    "lks_gradient_step_dev": (C.c_int, [C.c_int64, C.c_double, _P, _P, C.c_double, C.c_double, _P]),
    "lks_motion_filter_dev": (C.c_int, [_P, _P, _P, _P]),
    "lks_motion_filter_T_dev": (C.c_int, [_P, _P, _P, _P]),
    "lks_interp_positions_dev": (C.c_int, [_P, _P, _P, _P, _P]),
    "lks_interp_positions_T_dev": (C.c_int, [_P, _P, _P, _P, _P]),
    "lks_get_state": (C.c_int, [_P, _D, _D]),
    "lks_set_initial_state": (C.c_int, [_P, _D, _D]),
    "lks_set_adjoint_terminal": (C.c_int, [_P, _D, _D]),
    "lks_get_adjoint_initial": (C.c_int, [_P, _D, _D]),
    "lks_density_filter": (C.c_int, [_P, _D, _D]),
    "lks_density_filter_T": (C.c_int, [_P, _D, _D]),
    "lks_projection": (C.c_int, [C.c_int64, C.c_double, C.c_double, _D, _D, _D]),
    "lks_motion_filter": (C.c_int, [_P, _D, _D]),
    "lks_motion_filter_T": (C.c_int, [_P, _D, _D]),
    "lks_interp_positions": (C.c_int, [_P, _D, _D, _D]),
    "lks_interp_positions_T": (C.c_int, [_P, _D, _D, _D]),
    "lks_get_step_sensitivities": (C.c_int, [_P, _D, _D]),
    "lks_get_objective_terms": (C.c_int, [_P, _D, _D]),
    "lks_get_stats": (C.c_int, [_P, C.POINTER(lks_stats)]),
    "lks_get_status": (C.c_int, [_P]),
    "lks_set_angle_knots": (C.c_int, [_P, _D]),
    "lks_get_angle_gradient": (C.c_int, [_P, _D]),
    "lks_get_step_angle_sensitivities": (C.c_int, [_P, _D, _D]),
    "lks_get_angles": (C.c_int, [_P, _D, _D]),
    "lks_angles_T": (C.c_int, [_P, _D, _D, _D]),
    "lks_set_timing": (C.c_int, [_P, C.c_int]),
    "lks_set_graphs": (C.c_int, [_P, C.c_int]),
    "lks_batch_create": (C.c_int, [C.c_int, C.POINTER(lks_params), C.POINTER(_P)]),
    "lks_batch_destroy": (None, [_P]),
    "lks_batch_context": (_P, [_P, C.c_int]),
    "lks_batch_last_error": (C.c_char_p, [_P]),
    "lks_batch_forward_dev": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), _P, _P]),
    "lks_batch_adjoint_dev": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), _P]),
    "lks_density_filter_noalloc": (C.c_int, [C.POINTER(C.c_int32), C.c_double, _P, _P, _P]),
    "lks_noalloc_last_error": (C.c_char_p, []),
}

_lib = None


def load():
    """Load liblks.so (built in-tree) and declare every prototype; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with `python -m paper_2608_01071_b300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
