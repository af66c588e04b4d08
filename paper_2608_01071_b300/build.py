"""Build the CUDA library liblks.so in-tree for sm_103a (B300) with nvcc.

Usage: python -m paper_2608_01071_b300.build   (or build() from Python).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# the host runtime and one translation unit per (lattice, precision) of step-kernel engines, compiled in parallel
SRC = [os.path.join(HERE, "csrc", f) for f in ("lks_api.cu", "lks_engine2d_f32.cu", "lks_engine2d_f64.cu",
                                                  "lks_engine3d_f32.cu", "lks_engine3d_f64.cu")]
DEPS = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + [os.path.join(ROOT, "include", "lks.h")]
LIB = os.path.join(HERE, "liblks.so")
OBJ_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def up_to_date(target, sources):
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(s) <= t for s in sources)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed ({r.returncode}):\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        print(r.stderr, file=sys.stderr)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date(LIB, SRC + DEPS):
        return LIB
    from concurrent.futures import ThreadPoolExecutor

    os.makedirs(OBJ_DIR, exist_ok=True)
    objs = [os.path.join(OBJ_DIR, os.path.basename(f)[:-3] + ".o") for f in SRC]
    cmds = [[nvcc(), *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), *extra, "-c", f, "-o", o]
            for f, o in zip(SRC, objs)]
    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for fut in [ex.submit(_run, c, verbose) for c in cmds]:
            fut.result()
    _run([nvcc(), *ARCH, "-shared", *objs, "-o", LIB + ".tmp", "-lcudart"], verbose)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
