#!/usr/bin/env python3
"""Throughput of the fused forward + adjoint lattice-kinetic-scheme sweep (G node-steps/s, "GLUPS").

One step = one lks_forward + one lks_adjoint of the whole workload (all steps of the hot path: filters,
Nt forward LKS steps with the fused rigid-body mapping and objective, the checkpointed reverse sweep with
recompute, the adjoint steps with shape/motion sensitivities, the chain rules).  value = nodes x Nt /
(device time of one step), whole job (sum over ranks for --gpus N: independent replicas, weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_01071_b300.workloads import draw_gamma, draw_knots, workload  # noqa: E402

# the largest single-GPU configuration: D3Q15 on 256x128x128 (4.19 M nodes, 67 MB per FP32 state, HBM-bound),
# 8000 steps, binomial checkpoints under a 40 GB budget
DEFAULT_WORKLOAD = "d3q15_256x128x128_fp32"
L2_BYTES = 126 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true", help="skip the plain FP64 GPU run (error of the FP32 path "
                    "at the full horizon, and the FP64 path's own throughput)")
    ap.add_argument("--nt", type=int, default=0, help="override the horizon (short runs for profiler captures)")
    ap.add_argument("--optimize", type=int, default=0, help="also run this many projected-gradient optimisation "
                    "iterations (gamma step 0.05, position step 0.5 cell, normalised) and report J and s/iteration")
    ap.add_argument("--phi-var", type=float, default=0.0, help="weight phi of the variance term of the objective "
                    "(J1 = E - phi V); 0 = the mean E alone")
    ap.add_argument("--objective", choices=["J1", "J2"], default="J1", help="J1 (Eq. objective1, the workload's "
                    "probe box) or J2 (Eq. objective2, the oar: F_L + 0.3 F_D with drag_span = the design's y extent)")
    ap.add_argument("--tile-rows", default="", help="force step-kernel variants instead of autotuning: F, F,A or "
                    "F,A,R (tile_rows codes of the forward sweep, the adjoint and the recomputation)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                smax.append(float(v[2]))
            except ValueError:
                continue
            for nme, val in zip(names, v[5:9]):
                if val.lower() == "active":
                    reasons.add(nme)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's time is the slowest rank's); identity without a process group."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, nodes, Nt, steps, seconds):
    """Whole-job G node-steps/s of `world` replicas that each ran `steps` forward+adjoint passes."""
    return world * nodes * Nt * steps / seconds / 1e9


# Source files of the step kernels: the shared helpers, plus one file per kernel family.
COMMON_SOURCES = ["lks_common.cuh", "lks_step_kernels.cuh"]


def kernel_variant(lattice, rows, kind):
    """(name, source files, steps per launch) of the step kernel that a tile_rows code selects.

    kind is "fwd" or "adj".  D2Q9: 1/2 row tiles, 3 two steps per launch on row tiles, 4/8/16 warp columns,
    32/64 vectorised warp columns.  D3Q15: 1 the generic shared-memory kernel, 8/16 z-marching, 32/64/96
    separable z-marching (planes x rows per block 16 x 8, 32 x 8, 16 x 16), 128/160/192 plane-pair separable
    (16, 32 or 64 planes per block; 192 adjoint only)."""
    if lattice == "D3Q15":
        if rows == 1:
            return f"{kind}_step_kernel", "lks_step_kernels.cuh", 1
        if rows >= 128:
            zb = {128: 16, 160: 32, 192: 64}[rows]
            return f"{kind}3p_kernel<ZB={zb}>", ["lks_step3s.cuh", "lks_tma.cuh", "lks_step3p.cuh"], 1
        if rows >= 32:
            zb, ty = {32: (16, 8), 64: (32, 8), 96: (16, 16)}[rows]
            return f"{kind}3s_kernel<ZB={zb},TY={ty}>", "lks_step3s.cuh", 1
        return f"{kind}3d_kernel<ZB={rows}>", "lks_step3d.cuh", 1
    if rows == 3:
        return f"{kind}2r2_kernel", "lks_step2r.cuh", 2
    if rows <= 2:
        return f"{kind}2r_kernel<RPT={rows}>", "lks_step2r.cuh", 1
    if rows >= 32:
        return f"{kind}2v_kernel<R={rows}>", "lks_step2v.cuh", 1
    return f"{kind}2d_kernel<R={rows}>", "lks_step2d.cuh", 1


def source_sha(files):
    import hashlib

    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2608_01071_b300", "csrc", f), "rb").read())
    return h.hexdigest()


def captured_traffic(workload_name, kernel, source):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of this workload, or None when there is
    no capture of that kernel or its sources changed since the capture.

    The summary holds lines `traffic_bytes_per_launch <kernel> <bytes> src <sha256 prefix>`, the hash taken
    over the shared step-kernel headers followed by the kernel's own header."""
    import re

    path = os.path.join(ROOT, "profiles", f"step_kernels_{workload_name}.md")
    if not os.path.exists(path):
        return None
    sha = source_sha(COMMON_SOURCES + (list(source) if isinstance(source, (list, tuple)) else [source]))
    for m in re.finditer(r"traffic_bytes_per_launch (\S+) (\d+) src ([0-9a-f]+)", open(path).read()):
        if m.group(1) == kernel and sha.startswith(m.group(3)):
            return int(m.group(2))
    return None


def objective_name(w):
    if w.get("objective", "J1") == "J2":
        return f"J2 = F_L + {w['w_D']:g} F_D (the Brinkman force on the design grid)"
    phi = w.get("phi_var", 0.0)
    return "E (mean of n.u over the probe box)" if phi == 0.0 else f"E - {phi:g} V (mean and variance of n.u)"


def bench_workload(args):
    """The named workload with the command line's objective settings."""
    w = dict(workload(args.workload), phi_var=args.phi_var)
    if args.objective == "J2":
        w = dict(w, objective="J2", phi_var=0.0, w_D=0.3, drag_span=float(w["design"][1]))
    return w


def node_count(w):
    return int(np.prod(w["shape"]))


def sample_steps_for(w):
    """Steps of the oracle's bounded sample: about 12 M node-steps (10-30 s of numpy FP64 on one core), 1 to 60."""
    return int(max(1, min(60, 12e6 // node_count(w))))


def sample_workload(w, sample_steps):
    """The workload's grid and seeded inputs over its first `sample_steps` steps.  The motion amplitude scales with the
    horizon so that body speeds stay those of the workload, and the probe box straddles the body's downstream edge
    (same cross-section as the workload's probe) so that J and its gradients are not zero after a few steps."""
    d = len(w["shape"])
    nde0 = w["design"][0] + 2 * w["margin"]
    edge = int((w["shape"][0] - 1) / 2.0 + (nde0 - 1) / 2.0)
    lo = (edge - 8,) + tuple(w["probe_lo"][1:d])
    hi = (edge + 8,) + tuple(w["probe_hi"][1:d])
    return dict(w, Nt=sample_steps, K=min(w["K"], 6), R_t=max(1.0, sample_steps / 4),
                amp=w["amp"] * sample_steps / w["Nt"], probe_lo=lo, probe_hi=hi)


def cpu_baseline(w, sample_steps=None, with_result=False):
    """The FP64 oracle, as it stands, on a bounded sample of the workload (see sample_workload).
    With `with_result`, also its (J, dJ/dgamma, dJ/dknots) for the gradient-error check."""
    import oracle as O  # test infrastructure: only this leg and --impl reference use it
    from tests.helpers import oracle_problem

    sample_steps = sample_steps or sample_steps_for(w)
    ws = sample_workload(w, sample_steps)
    P = oracle_problem(ws)
    gamma, knots = draw_gamma(ws), draw_knots(ws)
    t0 = time.perf_counter()
    res = O.gradient(P, gamma, knots)
    dt = time.perf_counter() - t0
    val = node_count(ws) * sample_steps / dt / 1e9
    cb = {"value": val, "unit": "G node-steps/s (fwd+adj)", "cores": 1, "kind": "oracle",
          "sample": f"{w['name']} grid and inputs, first {sample_steps} of {w['Nt']} steps, probe box at the body's "
                    f"downstream edge, forward + exact adjoint + chain rules, numpy FP64, {dt:.1f} s"}
    return (cb, res) if with_result else cb


def gradient_error(w, oracle_result, sample_steps=None):
    """The CUDA path's J and gradients on the oracle's sample against the oracle (relative errors), beside the
    tolerance the gradients are held to."""
    from paper_2608_01071_b300 import Solver

    sample_steps = sample_steps or sample_steps_for(w)
    ws = sample_workload(w, sample_steps)
    s = Solver.from_workload(ws)
    J = s.forward(draw_gamma(ws), draw_knots(ws))
    dg, dk = s.adjoint()
    s.close()
    Jo, dgo, dko = oracle_result
    rl2 = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))
    return {"sample": f"the cpu_baseline sample ({sample_steps} steps)",
            "J": {"oracle": Jo, "cuda": J, "rel_err": abs(J - Jo) / max(abs(Jo), 1e-300)},
            "dgamma_rel_l2": rl2(dg, dgo), "dknots_rel_l2": rl2(dk, dko),
            "tolerance": {"gradients_rel_l2": 1e-3 if w["precision"] == "fp32" else 1e-10}}


def fp64_comparison(w, gamma, knots, res32):
    """The plain FP64 GPU path on the same inputs over the full horizon: its throughput (one forward + adjoint, CUDA
    events on its stream) and the FP32 path's errors against it (J; final velocity, max relative; gradients,
    relative L2)."""
    import torch

    from paper_2608_01071_b300 import Solver

    w64 = dict(w, precision="fp64")
    s = Solver.from_workload(w64)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    J = s.forward(gamma, knots)
    dg, dk = s.adjoint()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, u = s.state()
    st = s.stats()
    s.close()
    J32, u32, dg32, dk32 = res32
    rl2 = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))
    return {"fp64_value": node_count(w) * w["Nt"] / (ms * 1e-3) / 1e9, "unit": "G node-steps/s (fwd+adj, host-pointer "
            "calls, copies included)", "fp64_tile_rows": [st["tile_rows_fwd"], st["tile_rows_rec"], st["tile_rows_adj"]],
            "horizon": w["Nt"], "J": {"fp32": J32, "fp64": J, "rel_err": abs(J32 - J) / max(abs(J), 1e-300)},
            "u_final_rel_max": float(np.max(np.abs(u32 - u)) / max(np.max(np.abs(u)), 1e-300)),
            "dgamma_rel_l2": rl2(dg32, dg), "dknots_rel_l2": rl2(dk32, dk),
            "tolerance": {"u_rel_max": 1e-4, "gradients_rel_l2": 1e-3}}


def l2_copy_gbs(dev):
    """Copy bandwidth of a 2 x 16 MB working set that stays in L2 (read + write bytes, torch copy, best of 5 runs of
    200 copies, CUDA events): the roof of the step kernels on grids whose states fit in L2."""
    import torch

    a = torch.ones(4 * 2**20, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    best = 0.0
    for _ in range(5):
        for _ in range(20):
            b.copy_(a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * a.numel() * 4 * 200 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = bench_workload(args)
    sample_steps = sample_steps_for(w)
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, sample_steps)
        if i >= args.warmup:
            times.append(cb)
    val = statistics.mean(t["value"] for t in times)
    line = {"impl": "reference", "metric": "fwd+adjoint LKS GLUPS", "value": val, "unit": "G node-steps/s (fwd+adj)",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "grid": list(w["shape"]), "design": list(w["design"]), "Nt": w["Nt"],
                       "sample_Nt": sample_steps, "objective": objective_name(w)},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": times[0]["sample"], "value": val,
                             "unit": "G node-steps/s (fwd+adj)"},
            "e2e": {"value": val, "unit": "G node-steps/s (fwd+adj)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_2608_01071_b300 import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")

    w = bench_workload(args)
    if args.nt > 0:  # shorter horizon, same body speed
        w = dict(w, Nt=args.nt, K=min(w["K"], max(2, args.nt // 4)), R_t=max(1.0, w["R_t"] * args.nt / w["Nt"]),
                 amp=w["amp"] * args.nt / w["Nt"])
    if args.tile_rows:
        codes = [int(v) for v in args.tile_rows.split(",")]
        w = dict(w, tile_rows=codes[0], tile_rows_adj=codes[1] if len(codes) > 1 else 0,
                 tile_rows_rec=codes[2] if len(codes) > 2 else 0)
    D = len(w["shape"])
    N = node_count(w)
    solver = Solver.from_workload(w)
    st0 = solver.stats()
    solver.set_timing(True)
    gamma, knots = draw_gamma(w), draw_knots(w)
    dev = torch.device("cuda", local)
    d_gamma = torch.tensor(np.ascontiguousarray(gamma.T), device=dev)
    d_knots = torch.tensor(knots, device=dev)
    d_J = torch.empty((), dtype=torch.float64, device=dev)
    d_dg = torch.empty_like(d_gamma)
    d_dk = torch.empty_like(d_knots)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 2**20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def step():
        solver.forward_dev(d_gamma, d_knots, d_J, stream=stream)
        solver.adjoint_dev(d_dg, d_dk, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    st_adj, st_rec, st_fwd, launches = [], [], [], 0
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed iterations (not inside the timed span)
        ev[i][0].record(stream)
        solver.forward_dev(d_gamma, d_knots, d_J, stream=stream)
        ev[i][1].record(stream)
        solver.adjoint_dev(d_dg, d_dk, stream=stream)
        ev[i][2].record(stream)
        s = solver.stats()
        st_adj.append((s["ms_adjoint_steps"], s["adjoint_steps"]))
        st_rec.append((s["ms_recompute_steps"], s["recompute_steps"]))
        st_fwd.append((s["ms_forward_steps"], s["forward_steps"]))
        launches += s["kernel_launches"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    ms = [a.elapsed_time(c) for a, _, c in ev]
    t_dev = sum(ms) / 1e3
    t_dev = max_over_ranks(t_dev, dist, dev)
    value = job_throughput(world, N, w["Nt"], args.steps, t_dev)
    # forward-only and adjoint-only (the adjoint includes the recomputation and the chain rules)
    t_fwd_call = max_over_ranks(sum(a.elapsed_time(b) for a, b, _ in ev) / 1e3, dist, dev)
    t_adj_call = max_over_ranks(sum(b.elapsed_time(c) for _, b, c in ev) / 1e3, dist, dev)

    # roofline of the step kernels from their live CUDA-event durations (spans recorded on the launching
    # streams); algorithmic bytes per node: forward reads and writes the (D+1)-component state, the adjoint reads
    # and writes lambda and reads the stored velocity, and reads lambda once more over the design footprint box
    s = 4 if w["precision"] == "fp32" else 8
    Fbn = 1
    hw = 1 if w["kernel"] == "linear" else 2
    for a in range(D):
        Fbn *= w["design"][a] + 2 * w["margin"] + 2 * hw - 1
    adj_bytes = N * (2 * (D + 1) + D) * s + Fbn * (D + 1) * s
    fwd_bytes = N * 2 * (D + 1) * s
    # the roof follows the working set: a step reads one state and writes another; when both fit in L2 the step
    # kernels never reach HBM and their roof is the measured L2 copy bandwidth
    state_mb = N * (D + 1) * s / 2**20
    l2_resident = 2 * N * (D + 1) * s <= L2_BYTES
    if l2_resident:
        bound, peak, peak_kind = "l2", l2_copy_gbs(dev), "measured L2 copy bandwidth (2 x 16 MB, torch copy)"
    else:
        bound = "hbm"
        peak, peak_kind = peaks()
    # spans (ms) and launches-worth of steps per kind: the forward sweep, the recomputation, the adjoint steps
    t_f, n_f = sum(a for a, _ in st_fwd), sum(n for _, n in st_fwd)
    t_r, n_r = sum(a for a, _ in st_rec), sum(n for _, n in st_rec)
    t_a, n_a = sum(a for a, _ in st_adj), sum(n for _, n in st_adj)

    def kernel_entry(kind, rows, step_bytes, t_ms, n_steps):
        name, src, per_launch = kernel_variant(w["lattice"], rows, kind)
        step_ms = t_ms / max(1, n_steps)
        gbs = step_bytes / (step_ms * 1e-3) / 1e9 if step_ms > 0 else 0.0
        return {"bound": bound, "kernel": name, "achieved": gbs, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": gbs / peak, "traffic": captured_traffic(w["name"], name, src),
                "bytes_per_launch": step_bytes * per_launch, "us_per_launch": step_ms * per_launch * 1e3,
                "steps_per_launch": per_launch, "_t": t_ms}

    # the forward-step kernel of the forward sweep and of the recomputation (one entry when they are the same
    # variant: its launches averaged over both, the sweep and recompute means listed), and the adjoint kernel
    entries = []
    if st0["tile_rows_rec"] == st0["tile_rows_fwd"] or n_r == 0:
        e = kernel_entry("fwd", st0["tile_rows_fwd"], fwd_bytes, t_f + t_r, n_f + n_r)
        e["us_per_step_forward_sweep"] = 1e3 * t_f / max(1, n_f)
        e["us_per_step_recompute"] = 1e3 * t_r / max(1, n_r)
        entries.append(e)
    else:
        e = kernel_entry("fwd", st0["tile_rows_fwd"], fwd_bytes, t_f, n_f)
        e["role"] = "forward sweep"
        entries.append(e)
        e = kernel_entry("fwd", st0["tile_rows_rec"], fwd_bytes, t_r, n_r)
        e["role"] = "recomputation (beside the adjoint chain)"
        entries.append(e)
    entries.append(kernel_entry("adj", st0["tile_rows_adj"], adj_bytes, t_a, n_a))
    if st0.get("pipelined"):
        # the recomputation and the adjoint steps run at the same time on two streams: their live launch durations
        # include the sharing, so their fractions understate each kernel alone; the path fraction measures the whole
        for e in entries:
            if e.get("role") != "forward sweep":
                e["concurrent"] = "the recomputation and the adjoint chain share the GPU (two streams)"
    tot = max(1e-30, sum(e["_t"] for e in entries))
    for e in entries:
        # shares of the summed kernel spans (recompute overlaps the adjoint on its own stream)
        e["share_of_kernel_time"] = e.pop("_t") / tot
    entries.sort(key=lambda e: -e["share_of_kernel_time"])
    # the whole path: algorithmic bytes of every forward, recompute and adjoint step over the device time
    path_bytes = (n_f + n_r) * fwd_bytes + n_a * adj_bytes
    path_gbs = path_bytes / t_dev / 1e9
    roof = dict(entries[0], other_kernels=entries[1:],
                path={"achieved": path_gbs, "frac": path_gbs / peak, "unit": "GB/s",
                      "bytes_per_step": path_bytes / args.steps,
                      "note": "algorithmic bytes of all step kernels (forward, recompute, adjoint) / device time"})
    l2_note = (f"512 MB buffer written between timed steps; a step touches two {state_mb:.1f} MB states, "
               + ("more than the 126 MB L2" if not l2_resident else "which stay L2-resident"))

    # end to end through the host-pointer C ABI (H2D of gamma and knots, D2H of J and both gradients)
    e2e_times = []
    for i in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J32 = solver.forward(gamma, knots)
        dg32, dk32 = solver.adjoint()
        e2e_times.append(time.perf_counter() - t0)
    _, u32 = solver.state()  # final state of the last forward (the reverse sweep leaves it in place)
    e2e = world * N * w["Nt"] / statistics.mean(e2e_times) / 1e9
    nd = int(np.prod(w["design"]))
    h2d = nd * 8 + w["K"] * D * 8
    d2h = 8 + nd * 8 + w["K"] * D * 8

    if rank == 0:
        line = {
            "metric": "fwd+adjoint LKS GLUPS", "value": value, "unit": "G node-steps/s (fwd+adj)",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if w["precision"] == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": w["name"], "lattice": w["lattice"], "grid": list(w["shape"]), "design": list(w["design"]),
                       "Nt": w["Nt"], "K": w["K"], "precision": w["precision"] + " state / f64 accumulators",
                       "checkpointing": w["ckpt"], "parallelism": f"replicas{world}",
                       "objective": objective_name(w), "l2": l2_note},
            "roofline": roof,
            "e2e": {"value": e2e, "unit": "G node-steps/s (fwd+adj)", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches * world),
            "tile_rows": {"forward": st0["tile_rows_fwd"], "recompute": st0["tile_rows_rec"],
                          "adjoint": st0["tile_rows_adj"]},
            "forward_only": {"value": job_throughput(world, N, w["Nt"], args.steps, t_fwd_call),
                             "unit": "G node-steps/s (lks_forward)"},
            "adjoint_only": {"value": job_throughput(world, N, w["Nt"], args.steps, t_adj_call),
                             "unit": "G node-steps/s (lks_adjoint, recomputation included)"},
            "clocks": clk,
            "wall_s": t_wall,
        }
        if args.optimize > 0:
            from paper_2608_01071_b300.optimize import optimize

            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, hist = optimize(solver, gamma, knots, iters=args.optimize, pos_bound=w["amp"])
            dt = time.perf_counter() - t0
            line["optimize"] = {"iters": args.optimize, "s_per_iter": dt / args.optimize, "J": hist,
                                "gamma_step": 0.05, "pos_step_cells": 0.5, "pos_bound_cells": w["amp"]}
        if not args.no_fp64_check and w["precision"] == "fp32":
            line["fp32_vs_fp64_gpu"] = fp64_comparison(w, gamma, knots, (J32, u32, dg32, dk32))
        if not args.no_cpu_baseline:
            line["cpu_baseline"], ores = cpu_baseline(w, with_result=True)
            line["grad_error_vs_oracle"] = gradient_error(w, (ores[0], ores[1], ores[2]))
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def shard_instances(sizes, rank, world):
    """Instances of a study for one rank: largest first, each to the rank with the fewest nodes so far (ties to the
    lower rank).  Every rank computes the same assignment; the shards partition the study."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def run_batched(args):
    """The batched parameter study: 32 uneven D2Q9 instances, forward + adjoint of all of them per step.  Under
    torchrun the instances are sharded over the ranks (independent problems: no collective on the data path), and
    the throughput counts the whole study over the slowest rank's time."""
    import torch

    from paper_2608_01071_b300 import Batch
    from paper_2608_01071_b300.workloads import batched_study

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    study = batched_study()
    nodes_all = sum(int(np.prod(w["shape"])) for w in study)
    ws = [study[i] for i in shard_instances([int(np.prod(w["shape"])) for w in study], rank, world)]
    b = Batch(ws)
    dev = torch.device("cuda", local)
    gam = [torch.tensor(np.ascontiguousarray(draw_gamma(w).T), device=dev) for w in ws]
    kn = [torch.tensor(draw_knots(w), device=dev) for w in ws]
    J = torch.empty(len(ws), dtype=torch.float64, device=dev)
    dg = [torch.empty_like(g) for g in gam]
    dk = [torch.empty_like(k) for k in kn]
    stream = torch.cuda.current_stream(dev)

    def step():
        b.forward_dev(gam, kn, J, stream=stream)
        b.adjoint_dev(dg, dk, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t = max_over_ranks(sum(ms) / 1e3, dist, dev)
    value = nodes_all * study[0]["Nt"] * args.steps / t / 1e9
    launches = max_over_ranks(sum(b.context_stats(i)["kernel_launches"] for i in range(len(ws))), dist, dev)
    tiles = sorted({(tuple(w["shape"]), b.context_stats(i)["tile_rows_fwd"], b.context_stats(i)["tile_rows_adj"])
                    for i, w in enumerate(ws)})
    if rank == 0:
        line = {"metric": "fwd+adjoint LKS GLUPS", "value": value, "unit": "G node-steps/s (fwd+adj)", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batched_study_32xD2Q9", "instances": len(study), "Nt": study[0]["Nt"],
                           "nodes_total": nodes_all, "modes": "11 shape / 11 motion / 10 joint",
                           "parallelism": f"instances sharded over {world} GPU(s) by node count",
                           "tiles": [list(x[0]) + [x[1], x[2]] for x in tiles]},
                "gpu_launches": int(launches * args.steps * world), "clocks": clk}
        print(json.dumps(line), flush=True)
    b.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_study":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
