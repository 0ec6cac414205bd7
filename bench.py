"""Benchmark of the batched rigid-body step (one JSON line on stdout).

Workload: the 4096-env apartment batch (uneven env sizes: U{4..48} objects +
a 10-body mobile manipulator, U{10..60} static boxes, 4 substeps x 20
coloured-PGS iterations, dt = 0.01 s), synthetic and seeded. A step is one
env-step of every env. `value` is env-steps/s of the fused persistent,
CUDA-graph-captured form with the state resident in HBM; the plain
one-launch-per-stage form is timed beside it, and `e2e` times the same step
through msh_step_host with pinned host buffers (copies in the timed region).

--impl reference times the CPU oracle on the host cores (a bounded sample of
envs per step) on the same metric.

Multi-GPU (torchrun): every rank steps its own 4096 envs (weak scaling, no
collective on the data path); the value is all ranks' env-steps over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/sec at 4096 envs (fwd and fwd+bwd) vs plain step; % HBM roofline"
# DRAM bytes (read + write) of one k_fused launch from an ncu capture, keyed by
# (config, envs, threads per env) and stored with the hash of the step kernel's
# sources it was captured on; a launch of any other build reports null.
FUSED_TRAFFIC = {(3, 4096, 16): ("f7de7dc6e7f021a9", 50.009856e6 + 12.298752e6)}
KERNEL_SOURCES = ("msh.cu", "msh_fused.cuh", "msh_fused16.cu", "msh_fused32.cu", "msh_stages.cuh", "msh_collide.cuh",
                  "msh_math.cuh")
WORKLOADS = {1: "falling spheres over static boxes", 2: "fixed-base arm and gripper at a counter",
             3: "apartment batch of uneven size with a mobile manipulator",
             4: "arm pushing a goal box on a table", 5: "scale batch, 32 objects and 50 static boxes per env",
             6: "apartment batch with drawer and fridge-door receptacles"}
UNIT = "env-steps/s"
# bytes per env-step the method must move when contacts stay on chip:
# per dynamic body state read + write + params, per static box, plane, per
# joint, per DoF target
B_BODY, B_STATIC, B_PLANE, B_JOINT, B_DOF = 52 + 52 + 32, 40, 16, 80, 4
# solver flops per row update (generic sequential-impulse row: J.v over four
# 3-blocks, the impulse, its clamp and four 3-block velocity updates)
FLOP_ROW = 55
ROWS = {0: 6, 1: 8, 2: 6}   # rows per revolute / prismatic / planar joint with drive


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def algorithmic(scene):
    """Algorithmic bytes per step of the whole batch."""
    nb, ns, nj = scene.env_counts()
    return int((B_BODY * nb + B_STATIC * ns + B_PLANE + B_JOINT * nj).sum() + B_DOF * scene.max_dof * scene.num_envs)


def row_count(scene, contact_count):
    jt = scene.joint_type
    joint_rows = sum(ROWS[int(t)] for t in jt)
    return int(3 * np.asarray(contact_count).sum() + joint_rows)


def kernel_hash() -> str:
    """Hash of the sources the fused step kernel is built from."""
    import hashlib
    h = hashlib.sha256()
    for n in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_13211_b300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def workload_config(args, scene, cfg):
    """The workload a line measures (identical in both arms)."""
    return {"workload": f"config{args.config}: {WORKLOADS.get(args.config, 'batch')}, {scene.num_envs} envs",
            "envs": scene.num_envs, "bodies": scene.num_bodies, "static_boxes": scene.num_statics,
            "joints": scene.num_joints, "dt": cfg.dt, "substeps": cfg.substeps, "iterations": cfg.iterations,
            "solver": "mass-split Jacobi" if cfg.mode == 1 else "coloured PGS",
            "l2": "GPU arm: flushed between timed steps (256 MB write); the CPU arm has no GPU cache"}


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, over the whole batch: the
    warm-up steps in one call, then the K timed steps in one call (each env
    runs its steps inside one OpenMP task)."""
    import oracle
    from paper_2412_13211_b300 import scenes
    if rank != 0:
        return
    scene, cfg = scenes.make_config(args.config, num_envs=args.envs)
    cfg = dataclasses.replace(cfg, mode=args.mode)
    tg = scene.target_walk(args.steps + args.warmup)
    threads = os.cpu_count() or 1
    st, _ = oracle.step(scene, cfg, scene.state(), tg[:args.warmup], args.warmup, "f32", threads=threads)
    t0 = time.perf_counter()
    oracle.step(scene, cfg, st, tg[args.warmup:], args.steps, "f32", threads=threads)
    dt = time.perf_counter() - t0
    value = scene.num_envs * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(args, scene, cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"all {scene.num_envs} envs x {args.steps} steps after {args.warmup} "
                                       f"warm-up steps, FP32 oracle, OpenMP over envs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(scene, cfg, budget_s=12.0):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: the whole batch for as many steps as fit in about `budget_s`."""
    import oracle
    threads = os.cpu_count() or 1
    tg = scene.target_walk(201)
    t0 = time.perf_counter()
    st, _ = oracle.step(scene, cfg, scene.state(), tg[:1], 1, "f32", threads=threads)
    one = time.perf_counter() - t0
    steps = int(max(1, min(200, budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.step(scene, cfg, st, tg[1:1 + steps], steps, "f32", threads=threads)
    dt = time.perf_counter() - t0
    return {"value": scene.num_envs * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"all {scene.num_envs} envs x {steps} steps (after one warm-up step), FP32, "
                      f"{dt:.1f} s of CPU time"}


def time_fwd_bwd(sim, scene, tg, horizon, k, stream, reps=2, threads_per_env=32):
    """env-steps/s of forward + backward through a differentiable rollout of
    `horizon` steps (step checkpointing every k): CUDA events around the whole
    forward and backward pass, after one untimed warm-up pass."""
    import torch
    from paper_2412_13211_b300.autograd import rollout
    dev = sim.device
    goal_body = np.where(scene.goal_body >= 0, scene.goal_body, np.diff(scene.body_off) - 1)
    idx = torch.as_tensor(scene.body_off[:-1] + goal_body, device=dev, dtype=torch.long)
    own = scene.goal_body >= 0
    goal_np = scene.pos[scene.body_off[:-1] + goal_body] + np.array([0.1, 0.0, 0.0], np.float32)
    goal_np[own] = scene.goal_pos[own]
    goal = torch.as_tensor(goal_np, device=dev)
    init = [torch.as_tensor(np.asarray(a, np.float32), device=dev) for a in scene.state()]
    mass0 = torch.as_tensor(np.asarray(scene.body_mass, np.float32), device=dev)
    if tg.shape[0] < horizon:
        raise ValueError(f"{tg.shape[0]} target rows for a {horizon}-step rollout")
    targets0 = tg[:horizon].contiguous()

    def once():
        st = [x.clone().requires_grad_(True) for x in init]
        mass = mass0.clone().requires_grad_(True)
        targets = targets0.clone().requires_grad_(True)
        out = rollout(sim, st, targets, mass, k)
        d = out[0][idx] - goal
        (d * d).sum().backward()
        return st[2].grad

    with torch.cuda.stream(stream):
        sim.set_exec("fused", threads_per_env, False)
        once()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            g = once()
        b.record(stream)
        stream.synchronize()
    ms = a.elapsed_time(b) / reps
    tape_bytes = sim.scratch_bytes
    return {"value": scene.num_envs * horizon / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms,
            "horizon": horizon, "checkpoint_every": k, "finite": bool(torch.isfinite(g).all().item()),
            "library_device_bytes": int(tape_bytes),
            "note": "forward (fused) + recorded re-run of each checkpoint segment + msh_backward per step"}


def time_labels(dev, stream, hbm_peak, n_traj=262144, steps=200, reps=5, cpu=True):
    """Event labeling (Appendix A.5) of a Pick batch: n_traj trajectories x steps
    records (force, cumulative collision force: FP32; flags: u8), inputs in HBM
    (larger than L2), CUDA events over `reps` launches; the oracle (Python) is
    timed on a 1000-trajectory sample of the same batch."""
    import torch
    from paper_2412_13211_b300 import labels as GL, trajectories as TR
    small = TR.make(GL.PICK, num=2048, steps=steps, seed=1)
    reps_tile = n_traj // 2048
    traj_np = {k: (np.tile(v, (1, reps_tile)) if v.ndim == 2 else np.tile(v, reps_tile)) for k, v in small.items()}
    traj = GL.to_device(traj_np, dev)
    rec = int(traj_np["length"].astype(np.int64).sum())            # records the scan reads (t >= 0 of each length)
    in_bytes = 9 * rec                                              # 4 force + 4 cumcol + 1 flags per record
    out_bytes = n_traj * (32 + 4 + 4 + 4)                          # events, count, label, length read
    with torch.cuda.stream(stream):
        for _ in range(2):
            GL.label_events(GL.PICK, traj, stream=stream)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            GL.label_events(GL.PICK, traj, stream=stream)
        b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b) / reps
    gbs = (in_bytes + out_bytes) / (ms / 1e3) / 1e9
    res = {"metric": "trajectories labeled/s", "value": n_traj / (ms / 1e3), "ms_per_launch": ms,
           "workload": f"Pick, {n_traj} trajectories x {steps} steps (lengths 60-100 %)",
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "algorithmic_bytes": in_bytes + out_bytes,
                        "note": "9 B per record read (force, cumcol, flags) + 44 B per trajectory written"}}
    if cpu:
        import oracle.labels as OL
        n_cpu = 1000
        sub = {k: (v[:, :n_cpu] if v.ndim == 2 else v[:n_cpu]) for k, v in traj_np.items()}
        t0 = time.perf_counter()
        OL.label_batch(OL.PICK, sub)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": n_cpu / dt, "unit": "trajectories/s", "cores": 1, "kind": "oracle",
                               "sample": f"{n_cpu} trajectories of the batch, Python oracle"}
    return res


def time_render(sim, scene, stream, hbm_peak, width=128, height=128, reps=10, cpu=True):
    """Depth cameras: two cameras per env (scene.camera_mounts), 128x128, at the
    batch's current state; CUDA events over `reps` renders; the oracle on 32 envs."""
    import torch
    body, pose = scene.camera_mounts()
    fov, near, far = np.pi / 2, 0.01, 10.0
    sim.set_cameras(body, pose, width, height, fov, near, far)
    out = torch.empty((scene.num_envs, body.shape[1], height, width), dtype=torch.float32, device=sim.device)
    with torch.cuda.stream(stream):
        for _ in range(3):
            sim.render_depth(out, stream=stream)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            sim.render_depth(out, stream=stream)
        b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b) / reps
    frames = scene.num_envs * body.shape[1]
    out_bytes = out.numel() * 4
    gbs = out_bytes / (ms / 1e3) / 1e9
    hit = float((out > 0).float().mean().item())
    res = {"metric": "depth images/s", "value": frames / (ms / 1e3), "ms_per_render": ms,
           "workload": f"{scene.num_envs} envs x {body.shape[1]} cameras x {width}x{height}",
           "pixels_hit": hit,
           "roofline_hbm": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                            "note": "output writes only (4 B per pixel); the kernel is bound by FP32 "
                                    "intersection arithmetic, see the profile summary"}}
    if cpu:
        import oracle
        n = 32
        sub = scene.subset(np.arange(n))
        st = [t.detach().cpu().numpy() for t in (sim.pos, sim.quat)]
        b0 = scene.body_off[n]
        t0 = time.perf_counter()
        oracle.render_depth(sub, st[0][:b0], st[1][:b0], body[:n], pose[:n], width, height,
                            float(np.float32(height * 0.5 / np.tan(float(np.float32(fov)) * 0.5))), near, far, "f32")
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": n * body.shape[1] / dt, "unit": "depth images/s", "cores": oracle.cores(),
                               "kind": "oracle", "sample": f"first {n} envs, brute force per pixel"}
    return res


def time_control(dev, stream, start, envs=4096, steps=20, warmup=3, width=128, height=128, cpu=True):
    """Control steps of the articulated-receptacle apartment batch (config 6):
    per sample, the controller turns a normalised action into PD targets, five
    100 Hz physics steps run under it (one CUDA graph), and the two depth
    cameras of every env render 128x128 (Sec. 4.2's benchmark loop: 20 Hz
    control, 100 Hz physics, 2 cameras). Seeded uniform actions in
    [-0.3, 0.3]. CUDA events per sample with an L2 flush between samples."""
    import torch
    from paper_2412_13211_b300 import autotune, scenes
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = scenes.make_config(6, num_envs=envs, env_start=start)
    spec = sc.controller_spec()
    sim = MshSim(sc, cfg, device=dev, exec_form="fused", use_graph=True)
    t0 = torch.as_tensor(sc.targets0).to(dev)
    tuning = autotune.tune(sim, t0, steps=3, warmup=2)
    sim.set_exec(*tuning["best"], True)
    init = tuple(t.clone() for t in (sim.pos, sim.quat, sim.linvel, sim.angvel))
    sim.set_controller(spec)
    body, pose = sc.camera_mounts()
    sim.set_cameras(body, pose, width, height, np.pi / 2, 0.01, 10.0)
    depth = torch.empty((sc.num_envs, body.shape[1], height, width), dtype=torch.float32, device=dev)
    acts = torch.as_tensor(sc.random_actions(warmup + steps, spec.action_dim, amp=0.3)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run(parts, k0, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        with torch.cuda.stream(stream):
            for i in range(n):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                if "ctrl" in parts:
                    sim.control_step(acts[k0 + i], stream=stream)
                if "render" in parts:
                    sim.render_depth(depth, stream=stream)
                ev[i][1].record(stream)
        stream.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    run(("ctrl", "render"), 0, warmup)
    ms = run(("ctrl", "render"), warmup, steps)
    status = sim.status()
    ms_ctrl = run(("ctrl",), 0, max(3, steps // 2))
    ms_render = run(("render",), 0, max(3, steps // 2))
    res = {"metric": "samples/s (control steps x envs, 2 depth cameras rendered per sample)",
           "value": sc.num_envs / (ms / 1e3), "ms_per_control_step": ms, "steps": steps,
           "physics_ms": ms_ctrl, "render_ms": ms_render,
           "physics_steps_per_sample": spec.steps_per_action, "form": list(tuning["best"]),
           "workload": f"config6 apartments with a drawer and a fridge door, {sc.num_envs} envs, "
                       f"{sc.num_bodies} bodies, {sc.num_statics} static boxes, {sc.num_joints} joints, "
                       f"{body.shape[1]} cameras x {width}x{height}, actions U[-0.3, 0.3]",
           "gpu_launches_per_sample": 1 + spec.steps_per_action * sim.launches_per_step + 1,
           "status_nonzero_envs": int((status != 0).sum())}
    if cpu:
        import oracle
        from oracle import control as K
        n = 64
        sub = sc.subset(np.arange(n))
        st = tuple(t[:sc.body_off[n]].cpu().numpy() for t in init)
        a = acts[0, :n].cpu().numpy()
        c0 = time.perf_counter()
        st2, _, _ = K.control_step(sub, cfg, spec, st, a, sub.targets0, "f32")
        oracle.render_depth(sub, st2[0], st2[1], body[:n], pose[:n], width, height,
                            float(np.float32(height * 0.5 / np.tan(float(np.float32(np.pi / 2)) * 0.5))), 0.01, 10.0,
                            "f32")
        dt = time.perf_counter() - c0
        res["cpu_baseline"] = {"value": n / dt, "unit": "samples/s", "cores": oracle.cores(), "kind": "oracle",
                               "sample": f"one control step (controller, 5 physics steps, 2 depth cameras) "
                                         f"of the first {n} envs"}
    sim.close()
    return res


def run_scale_form(args, dev, envs=16384, horizon=64, k=8):
    """Config 5 at full size: the fused step (autotuned, CUDA graph, L2 flushed
    between steps) and a differentiable 64-step rollout with a checkpoint every
    8 steps; peak device memory = the library's allocations (workspaces, tape,
    adjoint workspaces) + torch's peak."""
    import torch
    from paper_2412_13211_b300 import autotune, scenes
    from paper_2412_13211_b300.sim import MshSim
    torch.cuda.reset_peak_memory_stats(dev)
    sc, cfg = scenes.make_config(5, num_envs=envs)
    sim = MshSim(sc, cfg, device=dev, exec_form="fused", use_graph=True)
    tg = torch.as_tensor(sc.target_walk(max(horizon, args.warmup + args.steps))).to(dev)
    tuning = autotune.tune(sim, tg[0], steps=3, warmup=2)
    form, tpe = tuning["best"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            sim.step(tg[t], stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            sim.step(tg[args.warmup + i], stream=stream)
            ev[i][1].record(stream)
    stream.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    for t, s0 in zip((sim.pos, sim.quat, sim.linvel, sim.angvel), sc.state()):
        t.copy_(torch.as_tensor(np.asarray(s0, np.float32)).to(dev))
    fb = time_fwd_bwd(sim, sc, tg, horizon=horizon, k=k, stream=stream, reps=1,
                      threads_per_env=tpe if form == "fused" else 32)
    lib_bytes = int(sim.scratch_bytes)
    torch_peak = int(torch.cuda.max_memory_allocated(dev))
    status = sim.status()
    sim.close()
    return {"workload": f"config5: {WORKLOADS[5]}, {envs} envs, {sc.num_bodies} bodies, {sc.num_statics} static "
                        f"boxes, {sc.num_joints} joints",
            "forward": {"value": envs / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "form": [form, tpe],
                        "steps": args.steps, "l2": "flushed between timed steps"},
            "fwd_bwd": fb, "peak_device_bytes": {"library": lib_bytes, "torch_peak_allocated": torch_peak,
                                                 "total": lib_bytes + torch_peak},
            "status_nonzero_envs": int((status != 0).sum())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="msh", choices=["msh", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--mode", type=int, default=0, choices=[0, 1],
                    help="solver: 0 coloured PGS (the configurations' own), 1 mass-split Jacobi")
    ap.add_argument("--threads-per-env", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-report", action="store_true")
    ap.add_argument("--no-labels", action="store_true")
    ap.add_argument("--no-render", action="store_true")
    ap.add_argument("--no-control", action="store_true")
    ap.add_argument("--bwd-horizon", type=int, default=16)
    ap.add_argument("--profile-backward", action="store_true",
                    help="only a short fwd+bwd rollout of the 512-env differentiation workload (small case for ncu)")
    ap.add_argument("--scale-form", action="store_true",
                    help="only the scale form: 16384 envs of config 5, forward env-steps/s and a 64-step "
                         "forward+backward with checkpoints every 8 steps, with peak device memory")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2412_13211_b300 import scenes
    from paper_2412_13211_b300.sim import MshSim

    torch.cuda.set_device(local)
    if args.profile_backward:
        sc4, cfg4 = scenes.make_config(4, num_envs=512)
        sim4 = MshSim(sc4, cfg4, device=torch.device("cuda", local))
        tg4 = torch.as_tensor(sc4.target_walk(8)).cuda()
        r = time_fwd_bwd(sim4, sc4, tg4, horizon=8, k=8, stream=torch.cuda.Stream(), reps=1)
        print(json.dumps({"profile_backward": r}))
        return
    if args.scale_form:
        print(json.dumps({"scale_form": run_scale_form(args, torch.device("cuda", local))}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    from paper_2412_13211_b300 import replicas
    start, _ = replicas.env_range(args.envs, rank)
    scene, cfg = scenes.make_config(args.config, num_envs=args.envs, env_start=start)
    cfg = dataclasses.replace(cfg, mode=args.mode)
    from paper_2412_13211_b300 import autotune
    sim = MshSim(scene, cfg, device=dev, exec_form="fused", use_graph=True)
    total = args.warmup + args.steps
    # targets for the timed steps and for the differentiable rollout's horizon
    tg = torch.as_tensor(scene.target_walk(max(total, args.bwd_horizon))).to(dev)
    if args.threads_per_env:
        sim.set_exec("fused", args.threads_per_env, True)
        tuning = {"best": ("fused", args.threads_per_env), "ms": {}}
    else:
        tuning = autotune.tune(sim, tg[0], steps=3, warmup=2)
    form, tpe = tuning["best"]
    init = tuple(t.clone() for t in (sim.pos, sim.quat, sim.linvel, sim.angvel))
    det = sim.detect()
    rows = row_count(scene, det["contact_count"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.Stream(dev)

    def timed(step_fn, k0, n):
        """Per-step CUDA-event times on `stream`, with an L2 flush between steps."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        with torch.cuda.stream(stream):
            for i in range(n):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                step_fn(k0 + i)
                ev[i][1].record(stream)
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def fused_step(k):
        sim.step(tg[k], stream=stream)

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            fused_step(k)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with Clocks(local) as clk:
        ms = timed(fused_step, args.warmup, args.steps)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    t_step = float(np.mean(ms))
    t_tot = replicas.slowest(float(np.sum(ms)) / 1e3, device=dev)
    value = replicas.job_throughput(scene.num_envs, args.steps, t_tot, world)
    status = sim.status()

    # the same fused step with the contact report on (forces, robot collision
    # force, grasp test written every step)
    report = None
    if not args.no_report:
        sim.set_report(*scene.report_spec())
        with torch.cuda.stream(stream):
            for k in range(3):
                fused_step(args.warmup + k)
        stream.synchronize()
        n_rep = max(3, min(args.steps, 20))
        rms = timed(fused_step, args.warmup, n_rep)
        sim.clear_report()
        report = {"ms_per_step": float(np.mean(rms)), "overhead": float(np.mean(rms) / t_step - 1.0),
                  "steps": n_rep}

    # plain form (one launch per stage), same inputs
    plain = None
    if not args.no_plain:
        for t, s in zip((sim.pos, sim.quat, sim.linvel, sim.angvel), init):
            t.copy_(s)
        sim.set_exec("plain", 128, True)
        with torch.cuda.stream(stream):
            for k in range(args.warmup):
                fused_step(k)
        stream.synchronize()
        n_plain = max(3, min(args.steps, 20))
        pms = timed(fused_step, args.warmup, n_plain)
        plain = {"value": scene.num_envs / (np.mean(pms) / 1e3), "unit": UNIT, "ms_per_step": float(np.mean(pms)),
                 "launches_per_step": sim.launches_per_step, "steps": n_plain, "graph": True}
        sim.set_exec(form, tpe, True)

    # forward + backward: a differentiable rollout (checkpoint every 8 steps) of
    # the same batch, loss = squared goal distance of one object per env
    fwd_bwd = None
    if not args.no_backward:
        fwd_bwd = time_fwd_bwd(sim, scene, tg, horizon=args.bwd_horizon, k=8, stream=stream,
                               threads_per_env=tpe if form == "fused" else 32)
        sim.set_exec(form, tpe, True)
        # the differentiation workload: 512 envs, arm pushing a goal box, 64-step horizon
        sc4, cfg4 = scenes.make_config(4, num_envs=512, env_start=rank * 512)
        sim4 = MshSim(sc4, cfg4, device=dev)
        tg4 = torch.as_tensor(sc4.target_walk(64)).to(dev)
        fwd_bwd["differentiation_workload"] = time_fwd_bwd(sim4, sc4, tg4, horizon=64, k=8, stream=stream, reps=1)
        sim4.close()

    # end to end through the C ABI with pinned host buffers
    host = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory() for a in scene.state()]
    htg = torch.from_numpy(np.ascontiguousarray(scene.target_walk(total), np.float32)).pin_memory()
    for k in range(args.warmup):
        sim.step_host(*host, htg[k], stream=stream)
    n_e2e = max(3, min(args.steps, 50))
    t0 = time.perf_counter()
    for k in range(n_e2e):
        sim.step_host(*host, htg[args.warmup + k], stream=stream)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    h2d = 52 * scene.num_bodies + 4 * scene.num_envs * scene.max_dof
    d2h = 52 * scene.num_bodies

    hbm_peak, sm_max, peak_kind = peaks()
    labels = None if args.no_labels else time_labels(dev, stream, hbm_peak, cpu=rank == 0 and not args.no_cpu_baseline)
    render = None if args.no_render else time_render(sim, scene, stream, hbm_peak,
                                                     cpu=rank == 0 and not args.no_cpu_baseline)
    control = None if args.no_control else time_control(dev, stream, start, envs=args.envs,
                                                        cpu=rank == 0 and not args.no_cpu_baseline)
    bytes_step = algorithmic(scene)
    flops_step = FLOP_ROW * rows * cfg.substeps * cfg.iterations
    alu_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12     # FP32 FMA lanes x clock, TFLOP/s
    achieved_tf = flops_step / (t_step / 1e3) / 1e12
    achieved_gbs = bytes_step / (t_step / 1e3) / 1e9
    khash = kernel_hash()
    cap = FUSED_TRAFFIC.get((args.config, scene.num_envs, tpe)) if form == "fused" else None
    traffic = cap[1] if cap and cap[0] == khash else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, scene, cfg),
        "implementation": {"form": f"{form} (autotuned) + CUDA graph", "threads_per_env": tpe,
                           "workspace_bytes_per_env": sim.workspace_bytes,
                           "tuning_ms_per_step": {k: round(v, 4) for k, v in tuning["ms"].items()},
                           "contact_points": int(det["contact_count"].sum()), "rows_per_substep": rows,
                           "kernel_sources_hash": khash},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / alu_peak, "traffic": traffic,
                     "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                             "peak_kind": peak_kind, "algorithmic_bytes_per_step": bytes_step},
                     "note": f"FP32 peak = 148 SMs x 128 lanes x 2 x {sm_max:.0f} MHz (derived, not measured); "
                             f"achieved = {FLOP_ROW} flop x solver rows x substeps x iterations / fused-kernel step "
                             f"time; hbm = algorithmic bytes per step / step time against the measured copy "
                             f"bandwidth; traffic = ncu DRAM bytes of one launch of this exact kernel build "
                             f"(null when the sources changed since the capture)"},
        "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_step": bytes_step},
        "plain_step": plain, "contact_report": report, "event_labeling": labels, "depth_cameras": render,
        "control_wrapper": control,
        "fwd_bwd": fwd_bwd,
        "e2e": {"value": scene.num_envs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": n_e2e},
        "gpu_launches": args.steps * sim.launches_per_step,
        "status_nonzero_envs": int((status != 0).sum()),
        "device_memory": {"library_bytes": int(sim.scratch_bytes),
                          "torch_peak_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
                          "note": "library: the step's workspaces, tape and adjoint workspaces of the 4096-env "
                                  "handle; torch: state, targets, L2 flush buffer and the other legs' tensors"},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cfg)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
