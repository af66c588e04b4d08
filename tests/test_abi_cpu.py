"""C ABI checks that need no GPU: the library loads, exports every declared symbol, and validates input."""
import ctypes as C
import os
import re

import pytest

from paper_2608_01071_b300 import _abi
from paper_2608_01071_b300.workloads import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lks_[A-Za-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    lib = _abi.load()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.PROTOTYPES, n


def test_exports_nothing_undeclared():
    # the library's dynamic symbol table holds the declared C ABI and nothing else of its own
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    names = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert names == set(declared_functions()), sorted(names ^ set(declared_functions()))


def test_params_layout_matches():
    lib = _abi.load()
    p = _abi.lks_params()
    assert lib.lks_default_params(C.byref(p)) == 0
    assert p.size == C.sizeof(_abi.lks_params)


def test_validation_errors_without_gpu():
    from paper_2608_01071_b300.binding import params_from_workload
    lib = _abi.load()
    base = params_from_workload(workload("d2q9_96x48_fp64"))
    h = C.c_void_p()
    for mutate in [lambda p: setattr(p, "nu", -1.0), lambda p: setattr(p, "K", 1),
                   lambda p: setattr(p, "lattice", 7), lambda p: setattr(p, "size", 12),
                   lambda p: p.probe_hi.__setitem__(0, 500), lambda p: setattr(p, "tile_rows", 5),
                   lambda p: setattr(p, "tile_rows_adj", 4),  # adjoint variant without a forward one
                   lambda p: (setattr(p, "tile_rows", 4), setattr(p, "tile_rows_adj", 5)),  # no such variant
                   lambda p: setattr(p, "tile_rows_rec", 4),  # recompute variant without a forward one
                   lambda p: (setattr(p, "tile_rows", 32), setattr(p, "n", (C.c_int32 * 3)(95, 48, 1))),
                   lambda p: setattr(p, "phi_var", float("nan")), lambda p: setattr(p, "phi_var", float("inf")),
                   lambda p: setattr(p, "objective", 5),
                   lambda p: (setattr(p, "objective", _abi.LKS_OBJ_OAR), setattr(p, "drag_span", 0.0)),
                   lambda p: (setattr(p, "objective", _abi.LKS_OBJ_OAR), setattr(p, "drag_span", 9.0),
                              setattr(p, "phi_var", 1.0))]:
        p = _abi.lks_params.from_buffer_copy(base)
        mutate(p)
        assert lib.lks_create(C.byref(p), C.byref(h)) == _abi.LKS_EINVAL
        assert len(lib.lks_last_error_string(None)) > 0
    assert lib.lks_strerror(-5) == b"unstable forward sweep"
    assert lib.lks_forward(None, None, None, None) == _abi.LKS_EINVAL
    E, V = C.c_double(), C.c_double()
    assert lib.lks_get_objective_terms(None, C.byref(E), C.byref(V)) == _abi.LKS_EINVAL


def test_design_too_large_for_period():
    from paper_2608_01071_b300.binding import params_from_workload
    lib = _abi.load()
    p = params_from_workload(workload("d2q9_96x48_fp64"))
    p.nd[0] = 94
    h = C.c_void_p()
    assert lib.lks_create(C.byref(p), C.byref(h)) == _abi.LKS_EINVAL


def test_unknown_objective_is_rejected():
    from paper_2608_01071_b300.binding import params_from_workload
    with pytest.raises(ValueError):
        params_from_workload(dict(workload("d2q9_96x48_fp64"), objective="J3"))


def test_noalloc_rejects_oversize_before_any_device_call():
    # the size check comes first, so it runs without a GPU; the pointers are never used on rejection
    lib = _abi.load()
    for shape in ((2048, 1024, 1), (1 << 21, 1 << 21, 1 << 22), (1 << 30, 1 << 30, 1 << 30), (0, 4, 4)):
        nd = (C.c_int32 * 3)(*shape)
        rc = lib.lks_density_filter_noalloc(nd, 2.0, C.c_void_p(16), C.c_void_p(16), None)
        assert rc == _abi.LKS_EINVAL, shape
