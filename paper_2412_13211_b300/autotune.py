"""Autotuner for the batched step: picks the execution form (one launch per
stage, one per substep, or one persistent launch per step) and the threads
per env for a given batch by timing each candidate on the batch itself.

Tuning leaves the simulation state unchanged (it is saved and restored) and
caches the choice per batch signature.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

CANDIDATES = [("fused", 8), ("fused", 16), ("fused", 32), ("fused", 64), ("fused", 128), ("substep", 64),
              ("substep", 128), ("plain", 128)]
_cache: dict = {}


def signature(scene, cfg) -> str:
    nb, ns, nj = scene.env_counts()
    return json.dumps([scene.num_envs, int(nb.sum()), int(nb.max()), int(ns.sum()), int(ns.max()),
                       int(nj.sum()), cfg.substeps, cfg.iterations, cfg.mode, cfg.max_contacts, cfg.max_pairs])


def tune(sim, targets=None, candidates=CANDIDATES, steps: int = 5, warmup: int = 2, cache_file: str | None = None,
         use_graph: bool = True) -> dict:
    """Times every candidate (CUDA events, mean ms per step) and configures
    `sim` with the fastest. Returns {"best": (form, tpe), "ms": {...}}."""
    key = signature(sim.scene, sim.cfg)
    disk = {}
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            disk = json.load(f)
    if key in _cache or key in disk:
        res = _cache.get(key) or disk[key]
        sim.set_exec(res["best"][0], res["best"][1], use_graph)
        return res
    saved = [t.clone() for t in (sim.pos, sim.quat, sim.linvel, sim.angvel)]
    if targets is None:
        targets = sim.targets
    ms = {}
    for form, tpe in candidates:
        try:
            sim.set_exec(form, tpe, use_graph)
        except RuntimeError:
            continue
        for _ in range(warmup):
            sim.step(targets)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            sim.step(targets)
        b.record()
        torch.cuda.synchronize()
        ms[f"{form}/{tpe}"] = a.elapsed_time(b) / steps
        for t, s in zip((sim.pos, sim.quat, sim.linvel, sim.angvel), saved):
            t.copy_(s)
    best = min(ms, key=ms.get)
    form, tpe = best.split("/")
    res = {"best": (form, int(tpe)), "ms": ms}
    sim.set_exec(form, int(tpe), use_graph)
    sim.clear_status()
    _cache[key] = res
    if cache_file:
        disk[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_file)), exist_ok=True)
        with open(cache_file, "w") as f:
            json.dump(disk, f)
    return res
