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
SOURCES = [os.path.join(HERE, "csrc", n) for n in ("msh.cu", "msh_fused16.cu", "msh_fused32.cu", "msh_labels.cu", "msh_render.cu")]
DEPS = (glob.glob(os.path.join(HERE, "csrc", "*.cu")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
        + glob.glob(os.path.join(HERE, "csrc", "*.h"))
        + [os.path.join(ROOT, "include", "msh.h")])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: the only fused multiply-adds are explicit fmaf calls, so every
# execution form of the step computes bitwise identical results.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


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
    """Compiles the translation units in parallel, then links the shared object."""
    if not force and not stale(LIB, DEPS):
        return LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    tag = f".{os.getpid()}.tmp"
    objs = [os.path.join(LIB_DIR, os.path.basename(src) + tag + ".o") for src in SOURCES]
    procs = []
    try:
        for src, obj in zip(SOURCES, objs):
            cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append(subprocess.Popen(cmd))
        codes = [pr.wait() for pr in procs]
        bad = [src for src, c in zip(SOURCES, codes) if c != 0]
        if bad:
            raise subprocess.CalledProcessError(1, "nvcc -c " + " ".join(bad))
        tmp = LIB + tag
        subprocess.check_call([nvcc()] + ARCH + ["-shared"] + objs + ["-o", tmp])
        os.replace(tmp, LIB)
    finally:
        for pr in procs:
            if pr.poll() is None:
                pr.kill()
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
