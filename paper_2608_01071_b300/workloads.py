"""Seeded synthetic workloads shaped like the paper's examples (Sec. 4: 2D pump, 2D oar, 3D pump).

This module holds plain data and random-number draws only: grid sizes, physical parameters, probe boxes,
and the seeded design field gamma and motion knots.  It contains none of the method's arithmetic, and
both the CUDA path and the CPU oracle take its arrays as inputs.

Array conventions: ``gamma`` is indexed [x, y(, z)] over the inner design grid; ``knots`` has shape (K, d)
and holds body-centre offsets in analysis cells at the K knot times (knot k at the fraction k/(K-1) of
the horizon).  The flat C-ABI order (x fastest) of a design array ``g`` is ``g.T.ravel()``.
"""
from __future__ import annotations

import copy

import numpy as np

# One entry per workload.  Shapes are (nx, ny[, nz]); periodic[a] False means wall planes at 0 and n-1.
WORKLOADS = {
    # 2D plain method, FP64, full state storage (small case)
    "d2q9_96x48_fp64": dict(
        lattice="D2Q9", shape=(96, 48), periodic=(True, False), nu=0.02, design=(24, 24), margin=2,
        kappa_max=1.0, q=0.1, kernel="linear", Nt=400, K=20, R_t=100.0, filter_R=0.0, beta=0.0, eta=0.5,
        probe_lo=(72, 16), probe_hi=(88, 32), direction=(1.0, 0.0), precision="fp64", ckpt="full",
        ckpt_slots=0, motion="sine_noise", amp=8.0, seed=0),
    # 2D larger, FP32 state / FP64 accumulators, sqrt(N) checkpoints
    "d2q9_512x256_fp32": dict(
        lattice="D2Q9", shape=(512, 256), periodic=(True, False), nu=0.01, design=(128, 128), margin=2,
        kappa_max=1.0, q=0.1, kernel="linear", Nt=4000, K=100, R_t=1000.0, filter_R=2.0, beta=8.0, eta=0.5,
        probe_lo=(384, 96), probe_hi=(448, 160), direction=(1.0, 0.0), precision="fp32", ckpt="sqrt",
        ckpt_slots=0, motion="sinusoids", amp=32.0, seed=1),
    # 3D, FP32 state, binomial checkpoints with 16 slots
    "d3q15_128x64x64_fp32": dict(
        lattice="D3Q15", shape=(128, 64, 64), periodic=(True, False, False), nu=0.02, design=(48, 48, 48),
        margin=2, kappa_max=1.0, q=0.1, kernel="linear", Nt=2000, K=50, R_t=500.0, filter_R=1.5, beta=0.0,
        eta=0.5, probe_lo=(108, 24, 24), probe_hi=(124, 40, 40), direction=(1.0, 0.0, 0.0), precision="fp32",
        ckpt="revolve", ckpt_slots=16, motion="sinusoids", amp=16.0, seed=2),
    # 3D large, FP32 state / FP64 sensitivity accumulation, binomial checkpoints under a 40 GB budget
    "d3q15_256x128x128_fp32": dict(
        lattice="D3Q15", shape=(256, 128, 128), periodic=(True, False, False), nu=0.005, design=(96, 96, 96),
        margin=2, kappa_max=1.0, q=0.1, kernel="linear", Nt=8000, K=200, R_t=2000.0, filter_R=1.5, beta=0.0,
        eta=0.5, probe_lo=(192, 48, 48), probe_hi=(224, 80, 80), direction=(1.0, 0.0, 0.0), precision="fp32",
        ckpt="revolve", ckpt_slots=0, ckpt_bytes=40 * 2**30, motion="sinusoids", amp=13.0, seed=3),
    # HBM-sized 2D sizing run; the amplitude is 4 cells so that the body speed (~amp 2 pi / Nt) stays ~0.05
    "d2q9_4096x4096_fp32": dict(
        lattice="D2Q9", shape=(4096, 4096), periodic=(True, False), nu=0.02, design=(1024, 1024), margin=2,
        kappa_max=1.0, q=0.1, kernel="linear", Nt=500, K=20, R_t=125.0, filter_R=0.0, beta=0.0, eta=0.5,
        probe_lo=(2600, 1536), probe_hi=(2856, 2560), direction=(1.0, 0.0), precision="fp32", ckpt="sqrt",
        ckpt_slots=0, motion="sine_noise", amp=4.0, seed=5),
}


def workload(name: str, **overrides) -> dict:
    """A copy of a named workload with optional overrides (e.g. a shorter horizon for a parity case)."""
    w = copy.deepcopy(WORKLOADS[name])
    w.update(overrides)
    w["name"] = name
    return w


def draw_gamma(w: dict) -> np.ndarray:
    """gamma ~ U(0, 1) i.i.d. over the inner design grid."""
    rng = np.random.default_rng(w["seed"])
    return rng.uniform(0.0, 1.0, tuple(w["design"]))


def draw_knots(w: dict) -> np.ndarray:
    """Body-centre offsets (cells) at the K knots.

    "sine_noise": x-offset amp*sin(2 pi k / K) + N(0, 0.5^2), other axes 0.
    "sinusoids":  per axis a sum of 3 sinusoids a_m sin(2 pi m k/(K-1) + phi_m), a_m ~ U(0, amp/3),
                  phi_m ~ U(0, 2 pi).
    """
    rng = np.random.default_rng(w["seed"] + 1000)
    K, d = w["K"], len(w["shape"])
    k = np.arange(K, dtype=np.float64)
    out = np.zeros((K, d))
    if w["motion"] == "sine_noise":
        out[:, 0] = w["amp"] * np.sin(2.0 * np.pi * k / K) + rng.normal(0.0, 0.5, K)
    elif w["motion"] == "sinusoids":
        frac = k / (K - 1)
        for a in range(d):
            amps = rng.uniform(0.0, w["amp"] / 3.0, 3)
            phases = rng.uniform(0.0, 2.0 * np.pi, 3)
            for m in range(3):
                out[:, a] += amps[m] * np.sin(2.0 * np.pi * (m + 1) * frac + phases[m])
    else:
        raise ValueError(w["motion"])
    return out


def batched_study(seed: int = 4, count: int = 32):
    """Parameter study of independent D2Q9 instances of mixed sizes, viscosities and gradient modes."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 64), (256, 128), (384, 192), (512, 256)]
    modes = ["shape"] * 11 + ["motion"] * 11 + ["joint"] * 10
    out = []
    for i in range(count):
        shape = sizes[int(rng.integers(0, len(sizes)))]
        design = (shape[0] // 4, shape[1] // 4)
        nx, ny = shape
        w = dict(
            lattice="D2Q9", shape=shape, periodic=(True, False), nu=float(rng.uniform(0.005, 0.05)),
            design=design, margin=2, kappa_max=1.0, q=0.1, kernel="linear", Nt=2000, K=40, R_t=500.0,
            filter_R=0.0, beta=0.0, eta=0.5,
            probe_lo=(3 * nx // 4, 3 * ny // 8), probe_hi=(3 * nx // 4 + nx // 8, 5 * ny // 8),
            direction=(1.0, 0.0), precision="fp32", ckpt="sqrt", ckpt_slots=0, motion="sinusoids",
            amp=ny / 8.0, seed=seed * 100 + i, mode=modes[i % len(modes)], name=f"study_{i}")
        out.append(w)
    return out
