"""The allocation-free density filter against the regular one, through the C ABI.

Some callers cannot allocate device memory (their framework owns the pool, or an allocation in their loop
is not acceptable); lks_density_filter_noalloc serves them with a fixed device array as scratch.  This file
is collected last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2608_01071_b300 import Solver, _abi
from paper_2608_01071_b300.workloads import workload

pytestmark = pytest.mark.gpu


def test_noalloc_filter_matches_regular_filter_twice():
    import torch

    lib = _abi.load()
    rng = np.random.default_rng(7)
    cases = [((24, 24, 1), 2.0), ((13, 9, 7), 1.5)]
    for shape, R in cases:  # two calls in a row, the second on a different size
        w = workload("d2q9_96x48_fp64")
        if shape[2] > 1:
            w = dict(w, lattice="D3Q15", shape=(40, 30, 30), periodic=(True, False, False), design=shape,
                     probe_lo=(30, 5, 5), probe_hi=(35, 10, 10), direction=(1.0, 0.0, 0.0))
        else:
            w = dict(w, design=shape[:2])
        w = dict(w, filter_R=R)
        s = Solver.from_workload(w)
        x = torch.tensor(rng.uniform(0, 1, int(np.prod(shape))), device="cuda", dtype=torch.float64)
        ref = torch.empty_like(x)
        s.density_filter_dev(x, ref)
        out = torch.full_like(x, float("nan"))
        nd = (C.c_int32 * 3)(*shape)
        rc = lib.lks_density_filter_noalloc(nd, R, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), None)
        assert rc == 0, lib.lks_noalloc_last_error()
        torch.cuda.synchronize()
        s.close()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err <= 1e-12, err


def test_noalloc_rejects_oversize():
    import torch

    lib = _abi.load()
    x = torch.zeros(8, device="cuda", dtype=torch.float64)
    # one node over the limit, and extents whose product overflows 64 bits if formed before the check
    for shape in ((2048, 1024, 1), (1 << 21, 1 << 21, 1 << 22), (1 << 30, 1 << 30, 1 << 30)):
        nd = (C.c_int32 * 3)(*shape)
        rc = lib.lks_density_filter_noalloc(nd, 2.0, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None)
        assert rc == _abi.LKS_EINVAL, shape
        assert b"exceeds" in lib.lks_noalloc_last_error()
