"""ctypes front end of the C++ oracle (test infrastructure only).

`build()` compiles oracle/msh_oracle.cpp with g++ (-O3, OpenMP,
-ffp-contract=off so that FP32 collision results are bit-reproducible) into
oracle/_build/liboracle.so. `step()` advances a batch of envs in FP32 or FP64;
`detect()` returns the collision stage (AABBs, pairs, contacts, colouring) for
given poses.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msh_oracle.cpp")
_SOURCES = [_SRC, os.path.join(_HERE, "msh_raycast.cpp")]
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle if the shared object is missing or older than its source."""
    if (not force and os.path.exists(_OUT)
            and all(os.path.getmtime(_OUT) >= os.path.getmtime(f) for f in _SOURCES)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O3", "-std=c++17", "-march=x86-64-v2", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared"] + _SOURCES + ["-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class _Scene(C.Structure):
    _fields_ = [("num_envs", C.c_int32), ("body_off", C.c_void_p), ("static_off", C.c_void_p),
                ("joint_off", C.c_void_p), ("max_dof", C.c_int32), ("body_shape", C.c_void_p),
                ("body_dims", C.c_void_p), ("body_mass", C.c_void_p), ("static_pose", C.c_void_p),
                ("static_half", C.c_void_p), ("joint_type", C.c_void_p), ("joint_parent", C.c_void_p),
                ("joint_child", C.c_void_p), ("joint_dof", C.c_void_p), ("joint_frame_a", C.c_void_p),
                ("joint_frame_b", C.c_void_p), ("joint_gains", C.c_void_p), ("joint_limits", C.c_void_p)]


class _Cfg(C.Structure):
    _fields_ = [("dt", C.c_double), ("substeps", C.c_int32), ("iterations", C.c_int32),
                ("mode", C.c_int32), ("gravity", C.c_double * 3), ("friction", C.c_double),
                ("restitution", C.c_double), ("contact_offset", C.c_double), ("baumgarte", C.c_double),
                ("joint_baumgarte", C.c_double), ("slop", C.c_double), ("max_contacts", C.c_int32),
                ("max_pairs", C.c_int32)]


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        for name in ("oracle_step_f32", "oracle_step_f64"):
            fn = getattr(lib, name)
            fn.argtypes = [P, P, P, P, P, P, P, C.c_int, P, C.c_int]
            fn.restype = C.c_int
        for name in ("oracle_detect_f32", "oracle_detect_f64"):
            fn = getattr(lib, name)
            fn.argtypes = [P] * 15
            fn.restype = C.c_int
        lib.oracle_step_f64x.argtypes = [P, P, P, P, P, P, P, P, C.c_int, P, C.c_int]
        lib.oracle_step_f64x.restype = C.c_int
        lib.oracle_grad_f64.argtypes = [P, P, P, P, P, P, P, C.c_int, P, P, C.c_int, P, P, P, P, P, P, C.c_int]
        lib.oracle_grad_f64.restype = C.c_int
        lib.oracle_max_threads.restype = C.c_int
        lib.oracle_clip_cap_drops.restype = C.c_longlong
        lib.oracle_step_lambdas_f32.argtypes = [P] * 7 + [C.c_int, P, C.c_int]
        lib.oracle_step_lambdas_f32.restype = C.c_int
        for fn in (lib.oracle_vjp_f32, lib.oracle_vjp_f64):
            fn.argtypes = [P] * 22 + [C.c_int, P]
            fn.restype = C.c_int
        for fn in (lib.oracle_render_depth_f32, lib.oracle_render_depth_f64):
            fn.argtypes = [P, P, P, P, P, C.c_int]
            fn.restype = C.c_int
        for fn in (lib.oracle_step_report_f32, lib.oracle_step_report_f64):
            fn.argtypes = [P, P, P, P, P, P, P, C.c_int, P, C.c_int, P, P, P, P, P, P]
            fn.restype = C.c_int
        _lib = lib
    return _lib


def cores() -> int:
    return int(load().oracle_max_threads())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Keep:
    """Holds contiguous copies of the descriptor arrays alive for a call."""

    def __init__(self, scene):
        c = np.ascontiguousarray
        self.arrs = dict(
            body_off=c(scene.body_off, np.int32), static_off=c(scene.static_off, np.int32),
            joint_off=c(scene.joint_off, np.int32), body_shape=c(scene.body_shape, np.int32),
            body_dims=c(scene.body_dims, np.float32), body_mass=c(scene.body_mass, np.float32),
            static_pose=c(scene.static_pose, np.float32), static_half=c(scene.static_half, np.float32),
            joint_type=c(scene.joint_type, np.int32), joint_parent=c(scene.joint_parent, np.int32),
            joint_child=c(scene.joint_child, np.int32), joint_dof=c(scene.joint_dof, np.int32),
            joint_frame_a=c(scene.joint_frame_a, np.float32),
            joint_frame_b=c(scene.joint_frame_b, np.float32),
            joint_gains=c(scene.joint_gains, np.float32), joint_limits=c(scene.joint_limits, np.float32))
        s = _Scene()
        s.num_envs = scene.num_envs
        s.max_dof = scene.max_dof
        for k, v in self.arrs.items():
            setattr(s, k, v.ctypes.data)
        self.struct = s


def _cfg(cfg) -> _Cfg:
    c = _Cfg()
    c.dt = cfg.dt
    c.substeps = cfg.substeps
    c.iterations = cfg.iterations
    c.mode = cfg.mode
    for i in range(3):
        c.gravity[i] = cfg.gravity[i]
    c.friction = cfg.friction
    c.restitution = cfg.restitution
    c.contact_offset = cfg.contact_offset
    c.baumgarte = cfg.baumgarte
    c.joint_baumgarte = cfg.joint_baumgarte
    c.slop = cfg.slop
    c.max_contacts = cfg.max_contacts
    c.max_pairs = cfg.max_pairs
    return c


def step(scene, cfg, state, targets=None, nsteps: int = 1, precision: str = "f32", threads: int = 0):
    """Advances `state` = (pos, quat, linvel, angvel) by `nsteps` steps.

    targets: f32 [nsteps, E, max_dof] absolute joint targets (None = zeros).
    Returns (new_state, status[E]). The input arrays are not modified."""
    lib = load()
    dt = np.float32 if precision == "f32" else np.float64
    st = [np.ascontiguousarray(a, dtype=dt).copy() for a in state]
    E = scene.num_envs
    md = max(scene.max_dof, 1)
    if targets is None:
        targets = np.zeros((nsteps, E, md), np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.float32).reshape(-1, E, md)
    assert targets.shape[0] >= nsteps
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    fn = lib.oracle_step_f32 if precision == "f32" else lib.oracle_step_f64
    rc = fn(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]), _ptr(st[3]),
            _ptr(targets), int(nsteps), _ptr(status), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle step failed: {rc}")
    return tuple(st), status


class _ReportSpec(C.Structure):
    _fields_ = [("body_flags", C.c_void_p), ("fingers", C.c_void_p), ("target", C.c_void_p),
                ("grasp_min_force", C.c_double), ("grasp_max_angle_deg", C.c_double)]


@dataclass
class OracleReport:
    body_force: np.ndarray     # [B,3] net contact force on each body, last step (N)
    target_force: np.ndarray   # [E,3] force on the target from end-effector links
    finger_force: np.ndarray   # [E,2,3] force on each finger from the target
    robot_force: np.ndarray    # [E] cumulative robot collision force (N)
    grasped: np.ndarray        # [E]


def step_report(scene, cfg, state, targets, nsteps, body_flags, fingers, target, grasp_min_force=0.5,
                grasp_max_angle_deg=85.0, robot_force=None, precision: str = "f32", threads: int = 0):
    """`nsteps` steps with the contact report (forces of the last step; the robot
    collision force of every step added to `robot_force`, zeros if None).
    Returns (new_state, status[E], OracleReport)."""
    lib = load()
    dt = np.float32 if precision == "f32" else np.float64
    st = [np.ascontiguousarray(a, dtype=dt).copy() for a in state]
    E, B = scene.num_envs, scene.num_bodies
    md = max(scene.max_dof, 1)
    if targets is None:
        targets = np.zeros((nsteps, E, md), np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.float32).reshape(-1, E, md)
    flags = np.ascontiguousarray(body_flags, np.int32)
    fing = np.ascontiguousarray(fingers, np.int32).reshape(E, 2)
    tgt = np.ascontiguousarray(target, np.int32).reshape(E)
    spec = _ReportSpec(flags.ctypes.data, fing.ctypes.data, tgt.ctypes.data, float(grasp_min_force),
                       float(grasp_max_angle_deg))
    rep = OracleReport(np.zeros((B, 3), dt), np.zeros((E, 3), dt), np.zeros((E, 2, 3), dt),
                       np.zeros(E, dt) if robot_force is None else np.ascontiguousarray(robot_force, dt).copy(),
                       np.zeros(E, np.int32))
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    fn = lib.oracle_step_report_f32 if precision == "f32" else lib.oracle_step_report_f64
    rc = fn(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]), _ptr(st[3]), _ptr(targets),
            int(nsteps), _ptr(status), int(threads), C.byref(spec), _ptr(rep.body_force), _ptr(rep.target_force),
            _ptr(rep.finger_force), _ptr(rep.robot_force), _ptr(rep.grasped))
    if rc != 0:
        raise RuntimeError(f"oracle step_report failed: {rc}")
    return tuple(st), status, rep


class _RayScene(C.Structure):
    _fields_ = [("num_envs", C.c_int32), ("body_off", C.c_void_p), ("static_off", C.c_void_p),
                ("body_shape", C.c_void_p), ("body_dims", C.c_void_p), ("static_pose", C.c_void_p),
                ("static_half", C.c_void_p)]


class _Cams(C.Structure):
    _fields_ = [("ncam", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("focal", C.c_float),
                ("near_", C.c_float), ("far_", C.c_float), ("body", C.c_void_p), ("pose", C.c_void_p)]


def render_depth(scene, pos, quat, cam_body, cam_pose, width, height, focal, near, far, precision="f32",
                 threads: int = 0):
    """Depth images [E, ncam, H, W] (z-depth in m, 0 = no hit) of every env's
    cameras at poses (pos, quat); cam_body [E, ncam] env-local mount bodies
    (-1: world), cam_pose [E, ncam, 7] mount-local poses; focal in pixels."""
    lib = load()
    dt = np.float32 if precision == "f32" else np.float64
    E = scene.num_envs
    body = np.ascontiguousarray(cam_body, np.int32).reshape(E, -1)
    ncam = body.shape[1]
    pose = np.ascontiguousarray(cam_pose, np.float32).reshape(E, ncam, 7)
    keep = [np.ascontiguousarray(a) for a in (scene.body_off, scene.static_off, scene.body_shape, scene.body_dims,
                                              scene.static_pose, scene.static_half)]
    rs = _RayScene(E, *[_ptr(a) for a in keep])
    cams = _Cams(ncam, int(width), int(height), float(focal), float(near), float(far), _ptr(body), _ptr(pose))
    p = np.ascontiguousarray(pos, dt)
    q = np.ascontiguousarray(quat, dt)
    out = np.zeros((E, ncam, int(height), int(width)), dt)
    fn = lib.oracle_render_depth_f32 if precision == "f32" else lib.oracle_render_depth_f64
    rc = fn(C.byref(rs), _ptr(p), _ptr(q), C.byref(cams), _ptr(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle render failed: {rc}")
    return out


@dataclass
class OracleDetect:
    aabb_body: np.ndarray      # [B,6]
    aabb_static: np.ndarray    # [S,6]
    pair_count: np.ndarray     # [E]
    pairs: np.ndarray          # [E,max_pairs,2]
    contact_count: np.ndarray  # [E]
    contact_ids: np.ndarray    # [E,max_contacts,2]
    contact_geom: np.ndarray   # [E,max_contacts,10]  n, ra, rb, s0
    manifold_count: np.ndarray  # [E]
    colours: np.ndarray        # [J + E*max_pairs]
    ncolours: np.ndarray       # [E]
    status: np.ndarray         # [E]


def detect(scene, cfg, pos, quat, precision: str = "f32") -> OracleDetect:
    """Collision stage (AABB, broadphase, narrowphase, colouring) at the given poses."""
    lib = load()
    dt = np.float32 if precision == "f32" else np.float64
    pos = np.ascontiguousarray(pos, dtype=dt)
    quat = np.ascontiguousarray(quat, dtype=dt)
    E, B, S, J = scene.num_envs, scene.num_bodies, scene.num_statics, scene.num_joints
    P, K = cfg.max_pairs, cfg.max_contacts
    out = OracleDetect(
        aabb_body=np.zeros((B, 6), dt), aabb_static=np.zeros((S, 6), dt),
        pair_count=np.zeros(E, np.int32), pairs=np.full((E, P, 2), -1, np.int32),
        contact_count=np.zeros(E, np.int32), contact_ids=np.full((E, K, 2), -1, np.int32),
        contact_geom=np.zeros((E, K, 10), dt), manifold_count=np.zeros(E, np.int32),
        colours=np.full(J + E * P, -1, np.int32), ncolours=np.zeros(E, np.int32),
        status=np.zeros(E, np.int32))
    keep = _Keep(scene)
    c = _cfg(cfg)
    fn = lib.oracle_detect_f32 if precision == "f32" else lib.oracle_detect_f64
    rc = fn(C.byref(keep.struct), C.byref(c), _ptr(pos), _ptr(quat), _ptr(out.aabb_body),
            _ptr(out.aabb_static), _ptr(out.pair_count), _ptr(out.pairs), _ptr(out.contact_count),
            _ptr(out.contact_ids), _ptr(out.contact_geom), _ptr(out.manifold_count),
            _ptr(out.colours), _ptr(out.ncolours), _ptr(out.status))
    if rc != 0:
        raise RuntimeError(f"oracle detect failed: {rc}")
    return out


def loss_and_directional(scene, cfg, state, targets, nsteps, goal_body, goal_pos, dvel=None, dtargets=None,
                         dmass=None, threads: int = 0):
    """FP64 rollout loss sum_e |x_goal - goal|^2 per env and its directional
    derivatives by forward-mode dual numbers (at most 4 directions).

    dvel [K,B,6] (linear then angular velocity), dtargets [K,nsteps,E,max_dof],
    dmass [K,B]. Returns (loss [E], dloss [K,E], status [E])."""
    lib = load()
    E, B = scene.num_envs, scene.num_bodies
    md = max(scene.max_dof, 1)
    K = max(len(x) for x in (dvel, dtargets, dmass) if x is not None)
    assert 1 <= K <= 4
    st = [np.ascontiguousarray(a, dtype=np.float64) for a in state]
    tg = np.ascontiguousarray(targets, dtype=np.float32).reshape(-1, E, md)
    f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    dvel, dtargets, dmass = f64(dvel), f64(dtargets), f64(dmass)
    loss = np.zeros(E)
    dloss = np.zeros((K, E))
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    gb = np.ascontiguousarray(goal_body, dtype=np.int32)
    gp = np.ascontiguousarray(goal_pos, dtype=np.float64)
    rc = lib.oracle_grad_f64(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]), _ptr(st[3]),
                             _ptr(tg), int(nsteps), _ptr(gb), _ptr(gp), int(K), _ptr(dvel), _ptr(dtargets),
                             _ptr(dmass), _ptr(loss), _ptr(dloss), _ptr(status), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle grad failed: {rc}")
    return loss, dloss, status


def step_f64x(scene, cfg, state, targets, nsteps, mass=None, threads: int = 0):
    """FP64 rollout whose joint targets [nsteps,E,max_dof] and optional body
    masses [B] are taken in double (exact perturbations for finite
    differences). Returns (new_state, status)."""
    lib = load()
    E = scene.num_envs
    md = max(scene.max_dof, 1)
    st = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in state]
    tg = np.ascontiguousarray(np.zeros((nsteps, E, md)) if targets is None else targets,
                              dtype=np.float64).reshape(-1, E, md)
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    rc = lib.oracle_step_f64x(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]),
                              _ptr(st[3]), _ptr(tg), _ptr(m), int(nsteps), _ptr(status), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle step failed: {rc}")
    return tuple(st), status


def loss_value(scene, cfg, state, targets, nsteps, goal_body, goal_pos, mass=None, threads: int = 0):
    """FP64 loss per env after `nsteps` steps; targets [nsteps,E,max_dof] and
    optional masses [B] are taken in double (for finite differences)."""
    lib = load()
    E = scene.num_envs
    md = max(scene.max_dof, 1)
    st = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in state]
    tg = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, E, md)
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    rc = lib.oracle_step_f64x(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]),
                              _ptr(st[3]), _ptr(tg), _ptr(m), int(nsteps), _ptr(status), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle step failed: {rc}")
    L = np.zeros(E)
    for e in range(E):
        g = goal_body[e]
        if g >= 0:
            d = st[0][scene.body_off[e] + g] - np.asarray(goal_pos[e], np.float64)
            L[e] = d @ d
    return L, status


class _Decisions(C.Structure):
    _fields_ = [("delta", C.c_double), ("len_tol", C.c_double), ("kmax", C.c_int32), ("nfragile", C.c_void_p),
                ("fragile", C.c_void_p), ("fragile_site", C.c_void_p), ("fragile_choice", C.c_void_p),
                ("fragile_margin", C.c_void_p),
                ("flip_off", C.c_void_p), ("flip_idx", C.c_void_p)]


@dataclass
class OracleVJP:
    """Adjoints of one step's inputs for a seed on its output (all float64)."""
    pos: np.ndarray       # [B,3]
    quat: np.ndarray      # [B,4] (all four components, as the step reads them)
    linvel: np.ndarray    # [B,3]
    angvel: np.ndarray    # [B,3]
    targets: np.ndarray   # [E,max_dof]
    mass: np.ndarray      # [B]
    out: tuple            # the stepped state (pos, quat, linvel, angvel)
    status: np.ndarray    # [E]
    nfragile: np.ndarray = None   # [E] fragile decisions per env (when requested)
    fragile: list = None          # per env: the first `kmax` fragile decision indices
    fragile_site: list = None     # per env: the solver row of each (-1: joint limit or contact bias)
    fragile_choice: list = None   # per env: the natural outcome of each (1: clamp active)
    fragile_margin: list = None   # per env: the margin of each


def step_vjp(scene, cfg, state, targets, seed, precision: str = "f32", threads: int = 0, fragile: bool = False,
             flips=None, delta: float = 1e-4, len_tol: float = 1e-6, kmax: int = 16) -> OracleVJP:
    """One step from `state` with joint targets [E, max_dof], and the
    vector-Jacobian products of the seed (pos, quat, linvel, angvel adjoints of
    the stepped state, float64) with respect to the step's state, targets and
    body masses, by reverse mode. precision "f32": the FP32 oracle's primal
    arithmetic and branch decisions (adjoints in double); "f64": the FP64
    oracle's.

    fragile: also report, per env, the branch decisions taken within rounding
    of their thresholds (impulse clamps within `delta` of the update's
    magnitude, joint-limit errors and, after the first substep, contact
    separations within `len_tol` of a kink). flips: per env a list of
    decision indices to take the other way (the other one-sided piece)."""
    lib = load()
    dt = np.float32 if precision == "f32" else np.float64
    E, B = scene.num_envs, scene.num_bodies
    md = max(scene.max_dof, 1)
    st = [np.ascontiguousarray(a, dtype=dt) for a in state]
    tg = np.ascontiguousarray(np.zeros((E, md)) if targets is None else targets, dtype=dt).reshape(E, -1)
    if scene.max_dof > 0:
        assert tg.shape[1] == scene.max_dof
    w = [np.ascontiguousarray(a, dtype=np.float64) for a in seed]
    out = [np.zeros_like(a) for a in st]
    g = [np.zeros(a.shape, np.float64) for a in st]
    gtg = np.zeros((E, max(scene.max_dof, 1)), np.float64)
    gm = np.zeros(B, np.float64)
    status = np.zeros(E, np.int32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    dec = None
    nfr = frag = None
    if fragile or flips is not None:
        nfr = np.zeros(E, np.int32)
        frag = np.full((E, kmax), -1, np.int32)
        fsite = np.full((E, kmax), -1, np.int32)
        fchoice = np.zeros((E, kmax), np.int32)
        fmarg = np.zeros((E, kmax))
        off = idx = None
        if flips is not None:
            off = np.zeros(E + 1, np.int32)
            off[1:] = np.cumsum([len(f) for f in flips])
            idx = np.ascontiguousarray(np.concatenate([np.asarray(f, np.int32) for f in flips] + [np.zeros(1, np.int32)]))
        dec = _Decisions(float(delta), float(len_tol), int(kmax), nfr.ctypes.data, frag.ctypes.data,
                         fsite.ctypes.data, fchoice.ctypes.data, fmarg.ctypes.data,
                         None if off is None else off.ctypes.data, None if idx is None else idx.ctypes.data)
    fn = lib.oracle_vjp_f32 if precision == "f32" else lib.oracle_vjp_f64
    rc = fn(C.byref(keep.struct), C.byref(c), *[_ptr(a) for a in st], _ptr(tg), *[_ptr(a) for a in w],
            *[_ptr(a) for a in out], *[_ptr(a) for a in g], _ptr(gtg), _ptr(gm), _ptr(status), int(threads),
            None if dec is None else C.byref(dec))
    if rc != 0:
        raise RuntimeError(f"oracle vjp failed: {rc}")
    r = OracleVJP(g[0], g[1], g[2], g[3], gtg[:, :scene.max_dof], gm, tuple(out), status)
    if nfr is not None:
        r.nfragile = nfr
        r.fragile = [list(frag[e, :min(int(nfr[e]), kmax)]) for e in range(E)]
        r.fragile_site = [list(fsite[e, :min(int(nfr[e]), kmax)]) for e in range(E)]
        r.fragile_choice = [list(fchoice[e, :min(int(nfr[e]), kmax)]) for e in range(E)]
        r.fragile_margin = [list(fmarg[e, :min(int(nfr[e]), kmax)]) for e in range(E)]
    return r


def trajectory(scene, cfg, state, targets, nsteps, precision: str = "f32", threads: int = 0):
    """The states x_0 .. x_nsteps of a rollout, one oracle step at a time."""
    xs = [tuple(np.ascontiguousarray(a, np.float32 if precision == "f32" else np.float64) for a in state)]
    st = np.zeros(scene.num_envs, np.int32)
    for t in range(nsteps):
        nxt, s = step(scene, cfg, xs[-1], None if targets is None else targets[t:t + 1], 1, precision, threads)
        xs.append(nxt)
        st |= s
    return xs, st


def goal_seed(scene, x_pos, goal_body, goal_pos):
    """Adjoint of the final state for the loss sum_e |x_goal(e) - goal(e)|^2."""
    B = scene.num_bodies
    w = [np.zeros((B, 3)), np.zeros((B, 4)), np.zeros((B, 3)), np.zeros((B, 3))]
    for e in range(scene.num_envs):
        gb = int(goal_body[e])
        if gb >= 0:
            i = scene.body_off[e] + gb
            w[0][i] = 2.0 * (np.asarray(x_pos[i], np.float64) - np.asarray(goal_pos[e], np.float64))
    return w


def rollout_grad(scene, cfg, state, targets, nsteps, seed_final, precision: str = "f32", threads: int = 0):
    """Reverse-mode gradient of a rollout: the step adjoints chained backwards
    along the oracle's own trajectory. seed_final: the adjoint of the last
    state (or a callable of that state returning it). Returns (grad of the
    initial state (4 arrays), grad of targets [nsteps,E,max_dof], grad of the
    masses [B], the trajectory, status)."""
    xs, st = trajectory(scene, cfg, state, targets, nsteps, precision, threads)
    w = seed_final(xs[-1]) if callable(seed_final) else [np.asarray(a, np.float64) for a in seed_final]
    gtg = np.zeros((nsteps, scene.num_envs, scene.max_dof))
    gm = np.zeros(scene.num_bodies)
    for t in range(nsteps - 1, -1, -1):
        r = step_vjp(scene, cfg, xs[t], None if targets is None else targets[t], w, precision, threads)
        w = [r.pos, r.quat, r.linvel, r.angvel]
        gtg[t] = r.targets
        gm += r.mass
        st |= r.status
    return w, gtg, gm, xs, st


def step_lambdas(scene, cfg, state, targets=None, threads: int = 0):
    """One FP32 step and the impulses after every sweep, [E, substeps,
    iterations, 8 * Jmax + 3 * max_contacts] (joint k row r at 8 k + r, Jmax
    the largest env's joint count; contact point c row i at 8 Jmax + 3 c + i;
    unused slots are NaN). Returns (new_state, lambdas)."""
    lib = load()
    st = [np.ascontiguousarray(a, dtype=np.float32).copy() for a in state]
    E = scene.num_envs
    md = max(scene.max_dof, 1)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.float32).reshape(E, md)
    jmax = max(1, int(np.diff(scene.joint_off).max(initial=0)))
    rows = 8 * jmax + 3 * cfg.max_contacts
    lam = np.full((E, cfg.substeps, cfg.iterations, rows), np.nan, np.float32)
    keep = _Keep(scene)
    c = _cfg(cfg)
    rc = lib.oracle_step_lambdas_f32(C.byref(keep.struct), C.byref(c), _ptr(st[0]), _ptr(st[1]), _ptr(st[2]),
                                     _ptr(st[3]), _ptr(tg), int(jmax), _ptr(lam), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle step_lambdas failed: {rc}")
    return tuple(st), lam


def clip_cap_drops() -> int:
    """Outputs the box-box clipper's 8-vertex cap has dropped so far."""
    return int(load().oracle_clip_cap_drops())
