"""Failure detection on the host side of the CUDA path, without a GPU fault.

- A checkpoint plan larger than the device: lks_create returns LKS_ENOMEM before allocating anything.
- NaN in the design or the motion knots: the forward's stability check reports LKS_EUNSTABLE.
- The asynchronous adjoint does not wait for the forward's stability flag: after an unstable forward it returns
  LKS_OK and fills its outputs with NaN, lks_get_status reports LKS_EUNSTABLE, and the host-pointer adjoint
  returns LKS_EUNSTABLE with its outputs untouched.
- Two processes that share the tuner's file run the same step kernels and return the same bits.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import tiny_workload
from paper_2608_01071_b300 import LKSError, Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots, workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ENOMEM, EUNSTABLE = -2, -5


def test_plan_larger_than_device_is_enomem():
    import torch

    # every state of 5000 steps kept in FP64 on the 256x128x128 grid: about 670 GB
    w = workload("d3q15_256x128x128_fp32", precision="fp64", ckpt="full", Nt=5000, tile_rows=32)
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(LKSError) as e:
        Solver.from_workload(w)
    assert e.value.code == ENOMEM
    assert "free" in str(e.value)
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 256 * 2**20  # nothing was allocated and kept


@pytest.mark.parametrize("where", ["gamma", "knots"])
def test_nan_input_is_unstable(where):
    w = tiny_workload("D2Q9", precision="fp32")
    gamma, knots = draw_gamma(w), draw_knots(w)
    if where == "gamma":
        gamma[3, 4] = np.nan
    else:
        knots[2, 0] = np.nan
    s = Solver.from_workload(w)
    with pytest.raises(LKSError) as e:
        s.forward(gamma, knots)
    assert e.value.code == EUNSTABLE
    s.close()


def test_async_adjoint_reports_instability():
    import torch

    w = tiny_workload("D2Q9", precision="fp32", u_crit=1e-9)
    gamma, knots = draw_gamma(w), draw_knots(w)
    s = Solver.from_workload(w)
    dev = torch.device("cuda")
    d_gamma = torch.tensor(np.ascontiguousarray(gamma.T), device=dev)
    d_knots = torch.tensor(knots, device=dev)
    d_J = torch.empty((), dtype=torch.float64, device=dev)
    d_dg = torch.zeros_like(d_gamma)
    d_dk = torch.zeros_like(d_knots)
    s.forward_dev(d_gamma, d_knots, d_J)  # enqueued, no wait
    s.adjoint_dev(d_dg, d_dk)             # enqueued behind the forward, no wait
    torch.cuda.synchronize()
    assert torch.isnan(d_dg).all() and torch.isnan(d_dk).all()
    with pytest.raises(LKSError) as e:
        s.status()
    assert e.value.code == EUNSTABLE
    # the host-pointer adjoint of an unstable forward: an error, and the caller's arrays untouched
    s.forward_dev(d_gamma, d_knots, d_J)
    import ctypes as C

    dg = np.full(w["design"][::-1], 7.0)
    dk = np.full((w["K"], 2), 7.0)
    rc = s.lib.lks_adjoint(s.h, dg.ctypes.data_as(C.POINTER(C.c_double)), dk.ctypes.data_as(C.POINTER(C.c_double)))
    assert rc == EUNSTABLE
    assert np.all(dg == 7.0) and np.all(dk == 7.0)
    s.close()
    # a stable run clears the status
    s = Solver.from_workload(dict(w, u_crit=0.3))
    s.forward(gamma, knots)
    s.status()
    s.close()


_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from helpers import tiny_workload
from paper_2608_01071_b300 import Solver
from paper_2608_01071_b300.workloads import draw_gamma, draw_knots
w = tiny_workload("D3Q15", precision="fp32", shape=(44, 21, 19), ckpt="sqrt")
s = Solver.from_workload(w)
J = s.forward(draw_gamma(w), draw_knots(w))
dg, dk = s.adjoint()
st = s.stats()
np.savez({out!r}, J=J, dg=dg, dk=dk, rows=[st["tile_rows_fwd"], st["tile_rows_rec"], st["tile_rows_adj"]])
"""


def test_two_processes_same_bits(tmp_path):
    tune = tmp_path / "tune.txt"
    env = dict(os.environ, LKS_TUNE_FILE=str(tune))
    res = []
    for i in range(2):
        out = tmp_path / f"run{i}.npz"
        code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=str(out))
        subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=600)
        res.append(np.load(out))
    # the first process tuned and wrote its choices, the second read them
    assert tune.exists() and len(tune.read_text().splitlines()) == 1
    a, b = res
    assert list(a["rows"]) == list(b["rows"])
    assert a["J"] == b["J"]
    assert np.array_equal(a["dg"], b["dg"]) and np.array_equal(a["dk"], b["dk"])
