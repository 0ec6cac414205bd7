"""Builds libmsh.so (the CUDA library behind include/msh.h) for sm_103a.

The shared object is written in-tree to paper_2412_13211_b300/_lib/ so that it
travels with the repository. Rebuilt when missing or older than a source.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libmsh.so")
SOURCES = [os.path.join(HERE, "csrc", n) for n in ("msh.cu", "msh_labels.cu", "msh_render.cu")]
DEPS = (glob.glob(os.path.join(HERE, "csrc", "*.cu")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
        + glob.glob(os.path.join(HERE, "csrc", "*.h"))
        + [os.path.join(ROOT, "include", "msh.h")])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: the only fused multiply-adds are explicit fmaf calls, so every
# execution form of the step computes bitwise identical results.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-shared",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsh.so")


def stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale(LIB, DEPS):
        return LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + FLAGS + SOURCES + ["-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
