"""Tensor copies (TMA) of the D3Q15 plane-pair kernels.

A block whose raw region lies inside the grid in x and y fetches its planes by 4-D tensor copies issued by one
thread; the others (periodic seams, wall rows, ragged tails) by per-thread asynchronous copies.  The data moved is
the same, so the results equal those of the per-thread copies everywhere (LKS_NO_TMA=1) bit for bit, and the oracle
within the FP32 tolerances.  The copies complete on barriers whose waits are bounded in time: a diagnostic wait
that nothing completes (LKS_WAIT_PROBE=1) expires, and the call reports LKS_ETIMEOUT with the device still usable.
"""
import os

import numpy as np
import pytest

from test_gpu_parity import check, gpu_run
from helpers import tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.binding import LKSError
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots

pytestmark = pytest.mark.gpu


def with_env(env, fn):
    """fn() with the environment variables of `env` set (read by the library when a context is created)."""
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def pair_workload(fwd, adj, Nt=12):
    # 100 x 28 x 40: raw regions inside the grid for the blocks at x0 = 32, 64 and y0 = 8, 16; the blocks at x0 = 0
    # (periodic seam), x0 = 96 (ragged, 4 columns), y0 = 0 and 24 (walls, ragged) copy per thread; ragged z blocks
    return tiny_workload("D3Q15", precision="fp32", tile_rows=fwd, tile_rows_adj=adj, shape=(100, 28, 40),
                         design=(16, 8, 10), probe_lo=(70, 6, 10), probe_hi=(90, 22, 30), ckpt="sqrt", Nt=Nt)


@pytest.mark.parametrize("fwd,adj", [(128, 192), (160, 160)])
def test_tensor_copies_match_per_thread_copies_and_oracle(fwd, adj):
    w = pair_workload(fwd, adj)
    g, _ = check(w, 1e-5, 1e-4, 1e-3)
    assert g["stats"]["tile_rows_fwd"] == fwd and g["stats"]["tile_rows_adj"] == adj
    h = with_env({"LKS_NO_TMA": "1"}, lambda: gpu_run(w, draw_gamma(w), draw_knots(w)))
    assert g["J"] == h["J"]
    for k in ("p", "u", "dgamma", "dknots", "gs", "guG"):
        assert np.array_equal(g[k], h[k]), k


def test_expired_wait_reports_timeout():
    w = pair_workload(128, 192, Nt=4)
    gamma, knots = draw_gamma(w), draw_knots(w)

    def forward_code():
        s = Solver.from_workload(w)
        try:
            with pytest.raises(LKSError) as e:
                s.forward(gamma, knots)
            return e.value.code
        finally:
            s.close()

    assert with_env({"LKS_WAIT_PROBE": "1", "LKS_WAIT_NS": "20000"}, forward_code) == -6  # LKS_ETIMEOUT
    # the device stays usable: a new context computes what the per-thread copies compute
    a = gpu_run(w, gamma, knots)
    b = with_env({"LKS_NO_TMA": "1"}, lambda: gpu_run(w, gamma, knots))
    assert a["J"] == b["J"] and np.array_equal(a["dgamma"], b["dgamma"])
