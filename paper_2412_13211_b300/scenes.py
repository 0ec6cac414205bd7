"""Seeded synthetic scene descriptors for the batched rigid-body step.

This module is input construction only. It draws shapes, masses, initial
poses, static boxes, joint frames, drive gains and joint-target random walks
with a seeded NumPy PCG64 generator, and holds none of the step's arithmetic
(no integration, collision or constraint math). The CPU oracle and the CUDA
library both read the arrays it returns.

The five workloads follow the benchmark configurations of the batched
rigid-body step: a sphere drop, a fixed-base manipulator at a counter, an
apartment-like batch with uneven env sizes, a differentiation scene at a
table and a large apartment batch. The ManiSkill-HAB paper (Sec. 4.2)
measures on ReplicaCAD apartments with YCB objects and a Fetch robot; those
assets are not available, so these seeded primitives stand in for them.

Conventions (shared by both implementations):
  * z is up, SI units, quaternions are (w, x, y, z).
  * shape types: 0 sphere (r), 1 capsule (r, half segment length along local x),
    2 box (half extents x, y, z).
  * joint types: 0 revolute, 1 prismatic, 2 planar; the joint axis is the x axis
    of the joint frame (planar: the plane normal is the frame's z axis).
  * joint_parent == -1 means the world; frame_a is then given in world space.
  * Every env has a static ground plane z = 0 in addition to its static boxes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPHERE, CAPSULE, BOX = 0, 1, 2
REVOLUTE, PRISMATIC, PLANAR = 0, 1, 2
MODE_COLOURED, MODE_JACOBI = 0, 1
# controller kinds of a DoF column (the control wrapper's descriptor)
CTRL_HOLD, CTRL_DELTA, CTRL_ABS, CTRL_BASE_X, CTRL_BASE_Y, CTRL_BASE_YAW = 0, 1, 2, 3, 4, 5

_S2 = float(np.sqrt(0.5))
Q_ID = (1.0, 0.0, 0.0, 0.0)
# Orientation of a vertical robot link: its local x axis points along world +z.
Q_LINK = (_S2, 0.0, -_S2, 0.0)
# Joint frames in world space (the frame's x axis is the joint axis).
QW_AXIS_Z = Q_LINK                 # x axis -> world +z
QW_AXIS_Y = (_S2, 0.0, 0.0, _S2)   # x axis -> world +y
QW_AXIS_NY = (_S2, 0.0, 0.0, -_S2)  # x axis -> world -y
# The same frames written in the local frame of a vertical link
# (conj(Q_LINK) composed with the world frame; constants, checked in tests).
QL_AXIS_Z = (1.0, 0.0, 0.0, 0.0)
QL_AXIS_Y = (0.5, 0.5, 0.5, 0.5)
QL_AXIS_NY = (0.5, -0.5, 0.5, -0.5)

# A hanging link: its local x axis points along world -z.
Q_HANG = (_S2, 0.0, _S2, 0.0)


def _qmul(a, b):
    """Hamilton product, used only to express constant world frames in a
    link's initial local frame when building a scene."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return (aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
            aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw)


def _local_frame(q_body, q_world):
    return _qmul((q_body[0], -q_body[1], -q_body[2], -q_body[3]), q_world)


# Default drive gains (stiffness, damping, force limit) per DoF kind.
ARM_GAINS = (1000.0, 100.0, 200.0)
FINGER_GAINS = (1000.0, 100.0, 200.0)
BASE_GAINS = (1000.0, 200.0, 200.0)
LINK_RADIUS = 0.04
FINGER_HALF = (0.01, 0.005, 0.025)
FINGER_LIMITS = (0.0, 0.05)


@dataclass
class SolverCfg:
    """Step parameters (SI units)."""
    dt: float = 0.01
    substeps: int = 1
    iterations: int = 10
    mode: int = MODE_COLOURED
    gravity: tuple = (0.0, 0.0, -9.81)
    friction: float = 0.5
    restitution: float = 0.0
    contact_offset: float = 0.01
    baumgarte: float = 0.2
    joint_baumgarte: float = 0.2
    slop: float = 0.001
    max_contacts: int = 256
    max_pairs: int = 1024


@dataclass
class ControllerSpec:
    """Per-DoF-column controller descriptor, shared by every env of a scene
    (Sec. 4.1: joint delta-position control of the arm, base linear and
    angular velocity, actions normalised to [-1, 1]; Sec. 4.2: 100 Hz physics
    under 20 Hz control, i.e. 5 physics steps per action)."""
    action_dim: int
    kind: np.ndarray     # int32 [max_dof]  CTRL_*
    action: np.ndarray   # int32 [max_dof]  action column (-1 for CTRL_HOLD)
    scale: np.ndarray    # f32 [max_dof]    delta per action (DELTA) or speed per action (BASE_*)
    lo: np.ndarray       # f32 [max_dof]    target range
    hi: np.ndarray       # f32 [max_dof]
    yaw_dof: int         # the base's yaw column (-1: no base)
    steps_per_action: int = 5


@dataclass
class Scene:
    """A batch of environments as flat arrays with CSR offsets per env."""
    name: str
    num_envs: int
    body_off: np.ndarray      # int32 [E+1]
    static_off: np.ndarray    # int32 [E+1]
    joint_off: np.ndarray     # int32 [E+1]
    max_dof: int
    body_shape: np.ndarray    # int32 [B]
    body_dims: np.ndarray     # f32 [B,4]
    body_mass: np.ndarray     # f32 [B]
    static_pose: np.ndarray   # f32 [S,7]  position, quaternion
    static_half: np.ndarray   # f32 [S,3]
    joint_type: np.ndarray    # int32 [J]
    joint_parent: np.ndarray  # int32 [J]  env-local body index or -1 (world)
    joint_child: np.ndarray   # int32 [J]  env-local body index
    joint_dof: np.ndarray     # int32 [J]  first env-local DoF slot
    joint_frame_a: np.ndarray  # f32 [J,7] in parent frame (world if parent=-1)
    joint_frame_b: np.ndarray  # f32 [J,7] in child frame
    joint_gains: np.ndarray   # f32 [J,4]  stiffness, damping, force limit, 0
    joint_limits: np.ndarray  # f32 [J,2]  lower, upper (prismatic only)
    pos: np.ndarray           # f32 [B,3]
    quat: np.ndarray          # f32 [B,4]
    linvel: np.ndarray        # f32 [B,3]
    angvel: np.ndarray        # f32 [B,3]
    targets0: np.ndarray      # f32 [E,max_dof]
    dof_sigma: np.ndarray     # f32 [E,max_dof]  random-walk step std
    dof_lo: np.ndarray        # f32 [E,max_dof]
    dof_hi: np.ndarray        # f32 [E,max_dof]
    goal_body: np.ndarray     # int32 [E]  env-local body index or -1
    goal_pos: np.ndarray      # f32 [E,3]
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def num_bodies(self) -> int:
        return int(self.body_off[-1])

    @property
    def num_statics(self) -> int:
        return int(self.static_off[-1])

    @property
    def num_joints(self) -> int:
        return int(self.joint_off[-1])

    def env_counts(self):
        return (np.diff(self.body_off), np.diff(self.static_off),
                np.diff(self.joint_off))

    def report_spec(self):
        """Inputs of the contact report from the joint structure: robot links
        are the bodies that joints connect (bit 0), the fingers are the children
        of each env's first two prismatic joints, the end-effector links are
        the fingers and their parent (bit 1), the target is the goal body.
        Returns (body_flags [B], fingers [E,2], target [E])."""
        E = self.num_envs
        flags = np.zeros(self.num_bodies, np.int32)
        fingers = np.full((E, 2), -1, np.int32)
        for e in range(E):
            b0 = self.body_off[e]
            fing = []
            for g in range(self.joint_off[e], self.joint_off[e + 1]):
                for b in (self.joint_parent[g], self.joint_child[g]):
                    if b >= 0:
                        flags[b0 + b] |= 1
                if self.joint_type[g] == PRISMATIC and len(fing) < 2:
                    fing.append(int(self.joint_child[g]))
                    if self.joint_parent[g] >= 0:
                        flags[b0 + self.joint_parent[g]] |= 2
            for k, b in enumerate(fing):
                fingers[e, k] = b
                flags[b0 + b] |= 2
        return flags, fingers, np.asarray(self.goal_body, np.int32).copy()

    def camera_mounts(self):
        """Two depth cameras per env, standing in for the paper's head and arm
        RGB-D cameras (Sec. 4.2). Camera frames look along +x. Head camera: on
        the mobile base 1 m above its centre, or 0.6 m behind and 0.9 m above
        a fixed arm's first joint, pitched down 0.6 rad; without a robot, in
        the world at (-1.5, 0, 1.2) pitched down 0.5 rad. Arm camera: on the
        hand (the fingers' parent link), 6 cm off its axis at the tip, looking
        along the link; without a robot, at (0, -1.5, 1.2) facing +y.
        Returns (body [E, 2] env-local or -1, pose [E, 2, 7])."""
        E = self.num_envs
        body = np.full((E, 2), -1, np.int32)
        pose = np.zeros((E, 2, 7), np.float32)

        def pitch(a):
            return (np.cos(a / 2), 0.0, np.sin(a / 2), 0.0)
        for e in range(E):
            j0, j1 = self.joint_off[e], self.joint_off[e + 1]
            hand = -1
            for g in range(j0, j1):
                if self.joint_type[g] == PRISMATIC and self.joint_parent[g] >= 0:
                    hand = int(self.joint_parent[g])
                    break
            if j1 > j0 and self.joint_type[j0] == PLANAR:
                body[e, 0] = int(self.joint_child[j0])
                pose[e, 0] = (0.0, 0.0, 1.0) + pitch(0.6)
            elif j1 > j0:
                a = self.joint_frame_a[j0][:3]
                pose[e, 0] = (a[0] - 0.6, a[1], a[2] + 0.9) + pitch(0.6)
            else:
                pose[e, 0] = (-1.5, 0.0, 1.2) + pitch(0.5)
            if hand >= 0:
                g = self.body_off[e] + hand
                body[e, 1] = hand
                pose[e, 1] = (float(self.body_dims[g][1]), 0.0, 0.06, 1.0, 0.0, 0.0, 0.0)
            else:
                yaw = (np.cos(np.pi / 4), 0.0, 0.0, np.sin(np.pi / 4))
                p_ = pitch(0.5)
                w0, x0, y0, z0 = yaw
                w1, x1, y1, z1 = p_
                q = (w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1, w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
                     w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1, w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1)
                pose[e, 1] = (0.0, -1.5, 1.2) + q
        return body, pose

    def controller_spec(self, arm_delta: float = 0.1, base_speed: float = 1.0, base_turn: float = 1.5,
                        steps_per_action: int = 5) -> ControllerSpec:
        """The robot's action layout: one column per arm joint (delta position,
        `arm_delta` rad per action), one gripper column driving both fingers to
        an absolute opening in their range, and for a mobile base a linear
        (`base_speed` m/s) and an angular (`base_turn` rad/s) velocity column.
        Joints whose drive has no stiffness (the passive drawer and door) keep
        their targets. Every env must share one DoF layout."""
        E, D = self.num_envs, self.max_dof
        if E == 0 or D == 0:
            raise ValueError("the scene has no actuated joints")
        specs = []
        for e in range(E):
            kind = np.zeros(D, np.int32)
            act = np.full(D, -1, np.int32)
            scale = np.zeros(D, np.float32)
            arm, grip, yaw = [], [], -1
            for g in range(self.joint_off[e], self.joint_off[e + 1]):
                d, jt = int(self.joint_dof[g]), int(self.joint_type[g])
                if self.joint_gains[g][0] <= 0.0:
                    continue
                if jt == PLANAR:
                    kind[d:d + 3] = (CTRL_BASE_X, CTRL_BASE_Y, CTRL_BASE_YAW)
                    yaw = d + 2
                elif jt == REVOLUTE:
                    arm.append(d)
                elif jt == PRISMATIC and self.joint_parent[g] >= 0:
                    grip.append(d)
            for k, d in enumerate(arm):
                kind[d], act[d], scale[d] = CTRL_DELTA, k, arm_delta
            na = len(arm)
            for d in grip:
                kind[d], act[d] = CTRL_ABS, na
            A = na + (1 if grip else 0)
            if yaw >= 0:
                for d in (yaw - 2, yaw - 1):
                    act[d], scale[d] = A, base_speed
                act[yaw], scale[yaw] = A + 1, base_turn
                A += 2
            specs.append((A, kind, act, scale, yaw))
        A, kind, act, scale, yaw = specs[0]
        for s_ in specs[1:]:
            if s_[0] != A or s_[4] != yaw or not (np.array_equal(s_[1], kind) and np.array_equal(s_[2], act)):
                raise ValueError("envs differ in their DoF layout")
        lo, hi = self.dof_lo[0].copy(), self.dof_hi[0].copy()
        ctl = kind != CTRL_HOLD
        if not (np.all(self.dof_lo[:, ctl] == lo[ctl]) and np.all(self.dof_hi[:, ctl] == hi[ctl])):
            raise ValueError("envs differ in the ranges of their actuated DoFs")
        return ControllerSpec(action_dim=int(A), kind=kind, action=act, scale=scale, lo=lo, hi=hi,
                              yaw_dof=int(yaw), steps_per_action=int(steps_per_action))

    def random_actions(self, steps: int, action_dim: int, seed: int = 0, amp: float = 0.3) -> np.ndarray:
        """Seeded uniform actions in [-amp, amp], f32 [steps, E, action_dim]
        (the paper's random-action benchmark clips actions to [-0.3, 0.3])."""
        rng = np.random.Generator(np.random.PCG64(7_000_001 * (seed + 1) + self.seed))
        return rng.uniform(-amp, amp, size=(steps, self.num_envs, action_dim)).astype(np.float32)

    def state(self):
        """Fresh copies of the initial state arrays (pos, quat, linvel, angvel)."""
        return (self.pos.copy(), self.quat.copy(), self.linvel.copy(),
                self.angvel.copy())

    def target_walk(self, steps: int, seed: int = 0) -> np.ndarray:
        """Seeded Gaussian random walk of absolute joint targets, clipped to
        each DoF's range: f32 [steps, E, max_dof]."""
        rng = np.random.Generator(np.random.PCG64(1_000_003 * (seed + 1) + self.seed))
        out = np.empty((steps, self.num_envs, max(self.max_dof, 1)), np.float32)
        if self.max_dof == 0:
            out[:] = 0.0
            return out
        cur = self.targets0.astype(np.float64).copy()
        for t in range(steps):
            cur = cur + self.dof_sigma * rng.standard_normal(cur.shape)
            cur = np.clip(cur, self.dof_lo, self.dof_hi)
            out[t] = cur
        return out

    def subset(self, envs) -> "Scene":
        """A scene holding only the listed envs (same per-env content)."""
        envs = np.asarray(envs, dtype=np.int64)
        bo, so, jo = self.body_off, self.static_off, self.joint_off

        def gather(off, arr):
            idx = np.concatenate([np.arange(off[e], off[e + 1]) for e in envs]) \
                if len(envs) else np.zeros(0, np.int64)
            return arr[idx]

        def offs(off):
            cnt = np.array([off[e + 1] - off[e] for e in envs], np.int64)
            return np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)

        return Scene(
            name=self.name, num_envs=len(envs),
            body_off=offs(bo), static_off=offs(so), joint_off=offs(jo),
            max_dof=self.max_dof,
            body_shape=gather(bo, self.body_shape), body_dims=gather(bo, self.body_dims),
            body_mass=gather(bo, self.body_mass),
            static_pose=gather(so, self.static_pose), static_half=gather(so, self.static_half),
            joint_type=gather(jo, self.joint_type), joint_parent=gather(jo, self.joint_parent),
            joint_child=gather(jo, self.joint_child), joint_dof=gather(jo, self.joint_dof),
            joint_frame_a=gather(jo, self.joint_frame_a),
            joint_frame_b=gather(jo, self.joint_frame_b),
            joint_gains=gather(jo, self.joint_gains), joint_limits=gather(jo, self.joint_limits),
            pos=gather(bo, self.pos), quat=gather(bo, self.quat),
            linvel=gather(bo, self.linvel), angvel=gather(bo, self.angvel),
            targets0=self.targets0[envs], dof_sigma=self.dof_sigma[envs],
            dof_lo=self.dof_lo[envs], dof_hi=self.dof_hi[envs],
            goal_body=self.goal_body[envs], goal_pos=self.goal_pos[envs],
            seed=self.seed, meta=dict(self.meta))


# --------------------------------------------------------------------------
# Per-env builder
# --------------------------------------------------------------------------
def _yaw_quat(yaw):
    return (float(np.cos(0.5 * yaw)), 0.0, 0.0, float(np.sin(0.5 * yaw)))


class _Env:
    def __init__(self):
        self.bodies = []    # (shape, dims4, mass, pos3, quat4, linvel3, angvel3)
        self.statics = []   # (pose7, half3)
        self.joints = []    # dict
        self.dofs = []      # (target0, sigma, lo, hi)
        self.goal_body = -1
        self.goal_pos = (0.0, 0.0, 0.0)

    def body(self, shape, dims, mass, pos, quat=Q_ID, linvel=(0, 0, 0), angvel=(0, 0, 0)):
        d = list(dims) + [0.0] * (4 - len(dims))
        self.bodies.append((shape, d, mass, tuple(pos), tuple(quat), tuple(linvel), tuple(angvel)))
        return len(self.bodies) - 1

    def static(self, pos, half, quat=Q_ID):
        self.statics.append((tuple(pos) + tuple(quat), tuple(half)))

    def joint(self, jtype, parent, child, frame_a, frame_b, gains, limits, dofs):
        first = len(self.dofs)
        for d in dofs:
            self.dofs.append(d)
        self.joints.append(dict(type=jtype, parent=parent, child=child, fa=frame_a,
                                fb=frame_b, gains=tuple(gains) + (0.0,),
                                limits=tuple(limits), dof=first))


def _pack(name, envs, seed, meta=None) -> Scene:
    E = len(envs)
    nb = np.array([len(e.bodies) for e in envs], np.int64)
    ns = np.array([len(e.statics) for e in envs], np.int64)
    nj = np.array([len(e.joints) for e in envs], np.int64)
    max_dof = max([len(e.dofs) for e in envs] + [0])

    def off(c):
        return np.concatenate([[0], np.cumsum(c)]).astype(np.int32)

    bodies = [b for e in envs for b in e.bodies]
    statics = [s for e in envs for s in e.statics]
    joints = [j for e in envs for j in e.joints]
    f32 = np.float32

    def arr(items, fn, shape, dt=f32):
        if not items:
            return np.zeros((0,) + shape, dt)
        return np.array([fn(x) for x in items], dt).reshape((-1,) + shape)

    t0 = np.zeros((E, max_dof), f32)
    sg = np.zeros((E, max_dof), f32)
    lo = np.zeros((E, max_dof), f32)
    hi = np.zeros((E, max_dof), f32)
    for i, e in enumerate(envs):
        for k, (a, s, l, h) in enumerate(e.dofs):
            t0[i, k], sg[i, k], lo[i, k], hi[i, k] = a, s, l, h
    return Scene(
        name=name, num_envs=E, body_off=off(nb), static_off=off(ns), joint_off=off(nj),
        max_dof=int(max_dof),
        body_shape=arr(bodies, lambda b: b[0], (), np.int32),
        body_dims=arr(bodies, lambda b: b[1], (4,)),
        body_mass=arr(bodies, lambda b: b[2], ()),
        static_pose=arr(statics, lambda s: s[0], (7,)),
        static_half=arr(statics, lambda s: s[1], (3,)),
        joint_type=arr(joints, lambda j: j["type"], (), np.int32),
        joint_parent=arr(joints, lambda j: j["parent"], (), np.int32),
        joint_child=arr(joints, lambda j: j["child"], (), np.int32),
        joint_dof=arr(joints, lambda j: j["dof"], (), np.int32),
        joint_frame_a=arr(joints, lambda j: j["fa"], (7,)),
        joint_frame_b=arr(joints, lambda j: j["fb"], (7,)),
        joint_gains=arr(joints, lambda j: j["gains"], (4,)),
        joint_limits=arr(joints, lambda j: j["limits"], (2,)),
        pos=arr(bodies, lambda b: b[3], (3,)),
        quat=arr(bodies, lambda b: b[4], (4,)),
        linvel=arr(bodies, lambda b: b[5], (3,)),
        angvel=arr(bodies, lambda b: b[6], (3,)),
        targets0=t0, dof_sigma=sg, dof_lo=lo, dof_hi=hi,
        goal_body=np.array([e.goal_body for e in envs], np.int32),
        goal_pos=np.array([e.goal_pos for e in envs], f32).reshape(E, 3),
        seed=seed, meta=meta or {})


# --------------------------------------------------------------------------
# Robot: 7 revolute capsule links + 2 prismatic box fingers, optionally on a
# planar (x, y, yaw) mobile base.
# --------------------------------------------------------------------------
def _add_hanging_robot(env: _Env, rng, anchor):
    """Adds the arm hanging from world point `anchor` (links point down, joint
    axes alternate world z / world y) with the two fingers at its lower end.
    Returns (link lengths, z of the finger bottoms)."""
    walk_rad, walk_fing = 0.02, 0.001
    ax, ay, az = anchor
    parent, prev_len = -1, None
    z = az
    lengths = [float(rng.uniform(0.1, 0.4)) for _ in range(7)]
    for i, L in enumerate(lengths):
        m = float(rng.uniform(1.0, 3.0))
        link = env.body(CAPSULE, (LINK_RADIUS, 0.5 * L), m, (ax, ay, z - 0.5 * L), Q_HANG)
        qw = QW_AXIS_Z if i % 2 == 0 else QW_AXIS_Y
        ql = _local_frame(Q_HANG, qw)
        fa = (ax, ay, az) + qw if parent == -1 else (0.5 * prev_len, 0.0, 0.0) + ql
        env.joint(REVOLUTE, parent, link, fa, (-0.5 * L, 0.0, 0.0) + ql, ARM_GAINS, (0.0, 0.0),
                  [(0.0, walk_rad, -np.pi, np.pi)])
        parent, prev_len = link, L
        z -= L
    hand_bottom = z
    fz = hand_bottom - LINK_RADIUS - FINGER_HALF[2] - 0.01
    dz = fz - (hand_bottom + 0.5 * prev_len)     # world offset from the hand centre
    for side, qw in ((+1.0, QW_AXIS_Y), (-1.0, QW_AXIS_NY)):
        dy = side * 0.015
        f = env.body(BOX, FINGER_HALF, 0.1, (ax, ay + dy, fz))
        # world offset (0, dy, dz) in the hanging link's frame is (-dz, dy, 0)
        env.joint(PRISMATIC, parent, f, (-dz, dy, 0.0) + _local_frame(Q_HANG, qw), (0.0, 0.0, 0.0) + qw,
                  FINGER_GAINS, FINGER_LIMITS, [(0.0, walk_fing, FINGER_LIMITS[0], FINGER_LIMITS[1])])
    return lengths, fz - FINGER_HALF[2]


def _add_robot(env: _Env, rng, anchor, mobile_base: bool):
    """Adds the robot with its first joint at world point `anchor` (fixed base)
    or on a base box whose centre is at `anchor` (mobile base). The arm stands
    vertically; joint axes alternate world z / world y."""
    ax, ay, az = anchor
    walk_rad, walk_fing, walk_base = 0.02, 0.001, 0.005
    if mobile_base:
        bh = (0.25, 0.25, 0.1)
        base = env.body(BOX, bh, 30.0, (ax, ay, az))
        # planar joint: frame a = world frame at the base centre, normal +z
        env.joint(PLANAR, -1, base, (ax, ay, az) + Q_ID, (0.0, 0.0, 0.0) + Q_ID,
                  BASE_GAINS, (0.0, 0.0),
                  [(0.0, walk_base, -2.0, 2.0), (0.0, walk_base, -2.0, 2.0),
                   (0.0, walk_rad, -np.pi, np.pi)])
        parent = base
        z0 = az + bh[2] + 0.06
        # joint frame on the base (identity orientation at start): local offset
        fa_pos = (0.0, 0.0, bh[2] + 0.06)
    else:
        parent = -1
        z0 = az
        fa_pos = (ax, ay, az)
    prev_len = None
    z = z0
    for i in range(7):
        L = float(rng.uniform(0.1, 0.4))
        m = float(rng.uniform(1.0, 3.0))
        link = env.body(CAPSULE, (LINK_RADIUS, 0.5 * L), m, (ax, ay, z + 0.5 * L), Q_LINK)
        hinge_z = (i % 2 == 0)
        qw = QW_AXIS_Z if hinge_z else QW_AXIS_Y
        ql = QL_AXIS_Z if hinge_z else QL_AXIS_Y
        if parent == -1:
            fa = fa_pos + qw
        elif prev_len is None:
            fa = fa_pos + qw          # parent is the base box (identity orientation)
        else:
            fa = (0.5 * prev_len, 0.0, 0.0) + ql
        fb = (-0.5 * L, 0.0, 0.0) + ql
        env.joint(REVOLUTE, parent, link, fa, fb, ARM_GAINS, (0.0, 0.0),
                  [(0.0, walk_rad, -np.pi, np.pi)])
        parent, prev_len = link, L
        z += L
    # fingers above the hand: world offset from the hand centre (dx, dy, dz) maps
    # to the vertical link's local frame as (dz, dy, -dx).
    hand_top = z
    fz = hand_top + LINK_RADIUS + FINGER_HALF[2] + 0.01
    dz = fz - (hand_top - 0.5 * prev_len)
    for side, qw, ql in ((+1.0, QW_AXIS_Y, QL_AXIS_Y), (-1.0, QW_AXIS_NY, QL_AXIS_NY)):
        dy = side * 0.015
        f = env.body(BOX, FINGER_HALF, 0.1, (ax, ay + dy, fz))
        env.joint(PRISMATIC, parent, f, (dz, dy, 0.0) + ql, (0.0, 0.0, 0.0) + qw,
                  FINGER_GAINS, FINGER_LIMITS,
                  [(0.0, walk_fing, FINGER_LIMITS[0], FINGER_LIMITS[1])])


# --------------------------------------------------------------------------
# Object placement on axis-aligned surfaces
# --------------------------------------------------------------------------
class _Surfaces:
    """Axis-aligned rectangles (x0, x1, y0, y1, top z) with placed footprints."""

    def __init__(self):
        self.rects = []
        self.placed = []   # per rect: list of (x, y, rho)

    def add(self, x0, x1, y0, y1, z):
        self.rects.append((x0, x1, y0, y1, z))
        self.placed.append([])

    def place(self, rng, k, rho, keep_out, tries=40):
        x0, x1, y0, y1, z = self.rects[k]
        if x1 - x0 < 2 * rho or y1 - y0 < 2 * rho:
            return None
        for _ in range(tries):
            x = rng.uniform(x0 + rho, x1 - rho)
            y = rng.uniform(y0 + rho, y1 - rho)
            ok = all((x - px) ** 2 + (y - py) ** 2 > (rho + pr + 0.005) ** 2
                     for px, py, pr in self.placed[k])
            ok = ok and all((x - kx) ** 2 + (y - ky) ** 2 > (rho + kr) ** 2
                            for kx, ky, kr in keep_out)
            if ok:
                self.placed[k].append((x, y, rho))
                return x, y, z
        return None


def _random_object(rng, kinds, size_lo, size_hi, mass_fn):
    kind = kinds[int(rng.integers(len(kinds)))]
    m = float(mass_fn())
    if kind == BOX:
        h = tuple(float(v) for v in rng.uniform(0.5 * size_lo, 0.5 * size_hi, 3))
        return BOX, h, m, float(np.hypot(h[0], h[1])), h[2]
    if kind == CAPSULE:
        r = float(rng.uniform(0.5 * size_lo, min(0.04, 0.25 * size_hi)))
        hl = float(rng.uniform(0.005, max(0.006, 0.5 * size_hi - r)))
        return CAPSULE, (r, hl), m, hl + r, r
    r = float(rng.uniform(0.5 * size_lo, 0.5 * size_hi))
    return SPHERE, (r,), m, r, r


def _place_objects(env, rng, surf, n, kinds, size_lo, size_hi, mass_fn, keep_out,
                   floor_rect=None):
    """Places n objects resting on surfaces (random yaw). Surfaces are tried in
    random order; the floor rectangle is the fallback."""
    placed = 0
    guard = 0
    while placed < n:
        guard += 1
        if guard > 200 * (n + 1):
            raise RuntimeError("object placement failed")
        shape, dims, m, rho, hz = _random_object(rng, kinds, size_lo, size_hi, mass_fn)
        order = rng.permutation(len(surf.rects))
        spot = None
        for k in order:
            spot = surf.place(rng, int(k), rho, keep_out)
            if spot is not None:
                break
        if spot is None:
            continue
        x, y, z = spot
        yaw = float(rng.uniform(0, 2 * np.pi))
        q = Q_ID if shape == SPHERE else _yaw_quat(yaw)
        env.body(shape, dims, m, (x, y, z + hz), q)
        placed += 1


# --------------------------------------------------------------------------
# Configurations
# --------------------------------------------------------------------------
def _rng(cfg, env, seed):
    return np.random.Generator(np.random.PCG64(cfg * 1000 + env + 7919 * seed))


def _cfg1_env(rng):
    env = _Env()
    boxes = []
    for _ in range(4):
        h = rng.uniform(0.1, 0.4, 3)
        c = (float(rng.uniform(-0.5, 0.5)), float(rng.uniform(-0.5, 0.5)), float(h[2]))
        yaw = float(rng.uniform(0, 2 * np.pi))
        env.static(c, tuple(float(v) for v in h), _yaw_quat(yaw))
        boxes.append((c, h, yaw))
    spheres = []
    while len(spheres) < 8:
        r = float(rng.uniform(0.03, 0.08))
        m = float(rng.uniform(0.1, 1.0))
        p = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.2, 1.2) + r])
        ok = all(np.linalg.norm(p - q) > r + rq + 0.01 for q, rq in spheres)
        for c, h, yaw in boxes:
            # distance from p to the yawed box (2-D rotation into the box frame)
            dx, dy = p[0] - c[0], p[1] - c[1]
            lx = np.cos(yaw) * dx + np.sin(yaw) * dy
            ly = -np.sin(yaw) * dx + np.cos(yaw) * dy
            lz = p[2] - c[2]
            d = np.maximum(np.abs([lx, ly, lz]) - h, 0.0)
            if np.linalg.norm(d) < r + 0.01:
                ok = False
        if ok:
            spheres.append((p, r))
            env.body(SPHERE, (r,), m, tuple(float(v) for v in p))
    return env


def _cfg2_env(rng):
    env = _Env()
    top = 0.9
    xs, ys = (-0.6, 0.0, 0.6), (0.0, 0.6)
    for x in xs:
        for y in ys:
            env.static((x, y, 0.5 * top), (0.3, 0.3, 0.5 * top))
    base = (0.0, 0.3, top + 0.06)
    _add_robot(env, rng, base, mobile_base=False)
    surf = _Surfaces()
    surf.add(-0.88, 0.88, -0.28, 0.88, top)
    _place_objects(env, rng, surf, 12, (BOX, CAPSULE), 0.03, 0.15,
                   lambda: rng.uniform(0.05, 0.5), keep_out=[(base[0], base[1], 0.2)])
    return env


def _cfg4_env(rng):
    """Arm hanging over a table with its fingers 3 cm above the top, the goal
    box 5 mm beside the fingers (so the target walk pushes it), five more
    boxes elsewhere on the table, and a goal near the goal box."""
    env = _Env()
    top = 0.8
    env.static((0.0, 0.0, 0.5 * top), (0.6, 0.4, 0.5 * top))
    # lengths are drawn inside the builder; the anchor height follows from them,
    # so draw them first with the same generator state and rebuild
    state = rng.bit_generator.state
    lengths = [float(rng.uniform(0.1, 0.4)) for _ in range(7)]
    rng.bit_generator.state = state
    drop = sum(lengths) + LINK_RADIUS + 0.01 + 2 * FINGER_HALF[2]
    anchor = (0.0, 0.0, top + 0.03 + drop)
    _, finger_bottom = _add_hanging_robot(env, rng, anchor)
    first = len(env.bodies)
    h = tuple(float(v) for v in rng.uniform(0.02, 0.05, 3))
    h = (h[0], h[1], max(h[2], 0.035))        # tall enough to reach the fingers
    gx = FINGER_HALF[0] + 0.005 + h[0]
    env.body(BOX, h, float(rng.uniform(0.05, 0.5)), (gx, 0.0, top + h[2]))
    surf = _Surfaces()
    surf.add(-0.58, 0.58, -0.38, 0.38, top)
    _place_objects(env, rng, surf, 5, (BOX,), 0.04, 0.10,
                   lambda: rng.uniform(0.05, 0.5), keep_out=[(0.0, 0.0, 0.25)])
    env.goal_body = first
    g = env.bodies[first][3]
    env.goal_pos = (g[0] + float(rng.uniform(-0.1, 0.1)), g[1] + float(rng.uniform(-0.1, 0.1)), g[2])
    return env


DRAWER_GAINS = (0.0, 5.0, 100.0)   # a damper only (no spring): passive articulations
DRAWER_LIMITS = (0.0, 0.35)
DOOR_LIMITS = (0.0, 1.57)


def _add_receptacles(env, W, D, foot):
    """A kitchen cabinet with a drawer and a fridge with a door against the +y
    wall (the paper's articulated receptacles, Sec. 3.1): the drawer slides out
    of the cabinet's cavity on a prismatic joint (0-0.35 m), the door swings
    into the room on a vertical hinge at its right edge (0-1.57 rad). Both are
    passive (damped) joints. Uses 5 static boxes."""
    yw = 0.5 * D
    # cabinet x in [-1.2, -0.4], 0.6 deep, 0.8 high: side panels, top, bottom around a cavity
    x0, x1, y0 = -1.2, -0.4, yw - 0.6
    cx = 0.5 * (x0 + x1)
    env.static((x0 + 0.02, yw - 0.3, 0.4), (0.02, 0.3, 0.4))
    env.static((x1 - 0.02, yw - 0.3, 0.4), (0.02, 0.3, 0.4))
    env.static((cx, yw - 0.3, 0.79), (0.5 * (x1 - x0), 0.3, 0.01))
    env.static((cx, yw - 0.3, 0.35), (0.5 * (x1 - x0) - 0.04, 0.3, 0.02))
    # the drawer: a box in the cavity, front flush with the cabinet front
    dh = (0.5 * (x1 - x0) - 0.05, 0.28, 0.17)
    dc = (cx, y0 + dh[1], 0.35 + 0.02 + dh[2] + 0.01)
    drawer = env.body(BOX, dh, 2.0, dc)
    q_out = (np.cos(-np.pi / 4), 0.0, 0.0, np.sin(-np.pi / 4))        # joint axis (local x) = world -y
    env.joint(PRISMATIC, -1, drawer, dc + q_out, (0.0, 0.0, 0.0) + q_out, DRAWER_GAINS, DRAWER_LIMITS,
              [(0.0, 0.0, DRAWER_LIMITS[0], DRAWER_LIMITS[1])])
    foot.append((x0, x1, yw - 0.6 - 0.4, yw))                          # keep the drawer's path clear
    # fridge x in [0.4, 1.1], 0.6 deep, 1.8 high; the door in front of it
    fx0, fx1 = 0.4, 1.1
    env.static((0.5 * (fx0 + fx1), yw - 0.3, 0.9), (0.5 * (fx1 - fx0), 0.3, 0.9))
    hx = 0.5 * (fx1 - fx0)
    door_c = (0.5 * (fx0 + fx1), yw - 0.6 - 0.025, 0.9)
    door = env.body(BOX, (hx, 0.02, 0.85), 8.0, door_c)
    q_up = (np.cos(-np.pi / 4), 0.0, np.sin(-np.pi / 4), 0.0)          # hinge frame: local x = world z
    hinge = (fx1, door_c[1], door_c[2])
    env.joint(REVOLUTE, -1, door, hinge + q_up, (hx, 0.0, 0.0) + q_up, DRAWER_GAINS, DOOR_LIMITS,
              [(0.0, 0.0, DOOR_LIMITS[0], DOOR_LIMITS[1])])
    foot.append((fx0 - 0.1, fx1 + 0.1, yw - 0.6 - 0.8, yw))           # the door's swing


def _apartment_env(rng, n_obj, n_static, kinds, size_lo, size_hi, mass_fn, receptacles=False):
    """A rectangular room (3-6 m sides) with four walls, counters and shelves
    along the walls, island counters when the walls are full, objects resting on
    furniture or the floor, and the mobile manipulator near the room centre;
    with `receptacles`, a cabinet drawer and a fridge door (5 of the statics)."""
    env = _Env()
    W, D = float(rng.uniform(3, 6)), float(rng.uniform(3, 6))
    t, H = 0.1, 2.5
    env.static((0.0, -0.5 * D - 0.5 * t, 0.5 * H), (0.5 * W + t, 0.5 * t, 0.5 * H))
    env.static((0.0, 0.5 * D + 0.5 * t, 0.5 * H), (0.5 * W + t, 0.5 * t, 0.5 * H))
    env.static((-0.5 * W - 0.5 * t, 0.0, 0.5 * H), (0.5 * t, 0.5 * D, 0.5 * H))
    env.static((0.5 * W + 0.5 * t, 0.0, 0.5 * H), (0.5 * t, 0.5 * D, 0.5 * H))
    left = n_static - 4
    rb = (float(rng.uniform(-0.3, 0.3)), float(rng.uniform(-0.3, 0.3)))
    keep = [(rb[0], rb[1], 0.6)]
    surf = _Surfaces()
    foot = []   # furniture footprints (x0, x1, y0, y1)
    if receptacles:
        _add_receptacles(env, W, D, foot)
        left -= 5

    def counter(x0, x1, y0, y1, h=0.9):
        env.static((0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * h),
                   (0.5 * (x1 - x0), 0.5 * (y1 - y0), 0.5 * h))
        surf.add(x0 + 0.02, x1 - 0.02, y0 + 0.02, y1 - 0.02, h)
        foot.append((x0, x1, y0, y1))

    def shelf(x0, x1, y0, y1, along_x):
        # two side panels + three boards at 0.35, 0.75, 1.15 m
        if along_x:
            env.static((x0 + 0.01, 0.5 * (y0 + y1), 0.6), (0.01, 0.5 * (y1 - y0), 0.6))
            env.static((x1 - 0.01, 0.5 * (y0 + y1), 0.6), (0.01, 0.5 * (y1 - y0), 0.6))
            bx0, bx1, by0, by1 = x0 + 0.02, x1 - 0.02, y0, y1
        else:
            env.static((0.5 * (x0 + x1), y0 + 0.01, 0.6), (0.5 * (x1 - x0), 0.01, 0.6))
            env.static((0.5 * (x0 + x1), y1 - 0.01, 0.6), (0.5 * (x1 - x0), 0.01, 0.6))
            bx0, bx1, by0, by1 = x0, x1, y0 + 0.02, y1 - 0.02
        for z in (0.35, 0.75, 1.15):
            env.static((0.5 * (bx0 + bx1), 0.5 * (by0 + by1), z),
                       (0.5 * (bx1 - bx0), 0.5 * (by1 - by0), 0.01))
            surf.add(bx0 + 0.01, bx1 - 0.01, by0 + 0.01, by1 - 0.01, z + 0.01)
        foot.append((x0, x1, y0, y1))

    # walk the four walls placing furniture side by side
    for wall in range(4):
        along_x = wall < 2
        span = W if along_x else D
        pos = -0.5 * span + 0.05
        while left > 0:
            kind_shelf = left >= 5 and rng.uniform() < 0.5
            length = float(rng.uniform(0.6, 1.2) if kind_shelf else rng.uniform(0.6, 1.5))
            if pos + length > 0.5 * span - 0.05:
                break
            depth = 0.35 if kind_shelf else 0.6
            if along_x:
                x0, x1 = pos, pos + length
                if wall == 0:
                    y0, y1 = -0.5 * D, -0.5 * D + depth
                else:
                    y0, y1 = 0.5 * D - depth, 0.5 * D
            else:
                y0, y1 = pos, pos + length
                if wall == 2:
                    x0, x1 = -0.5 * W, -0.5 * W + depth
                else:
                    x0, x1 = 0.5 * W - depth, 0.5 * W
            # corners: skip a slot that overlaps furniture on the previous wall
            clash = any(x0 < f1 and f0 < x1 and y0 < g1 and g0 < y1 for f0, f1, g0, g1 in foot)
            if not clash:
                if kind_shelf:
                    shelf(x0, x1, y0, y1, along_x)
                    left -= 5
                else:
                    counter(x0, x1, y0, y1)
                    left -= 1
            pos += length + float(rng.uniform(0.05, 0.4))
    # island counters for the rest; once the floor is full, thin wall panels
    # mounted above furniture height (1.4-2.3 m), where no object is spawned
    tries = 0
    while left > 0 and tries < 400:
        tries += 1
        lx, ly = float(rng.uniform(0.3, 0.8)), float(rng.uniform(0.3, 0.8))
        cx = float(rng.uniform(-0.5 * W + lx, 0.5 * W - lx))
        cy = float(rng.uniform(-0.5 * D + ly, 0.5 * D - ly))
        x0, x1, y0, y1 = cx - 0.5 * lx, cx + 0.5 * lx, cy - 0.5 * ly, cy + 0.5 * ly
        clash = any(x0 < f1 + 0.1 and f0 < x1 + 0.1 and y0 < g1 + 0.1 and g0 < y1 + 0.1
                    for f0, f1, g0, g1 in foot)
        near = (cx - rb[0]) ** 2 + (cy - rb[1]) ** 2 < (0.9 + 0.5 * max(lx, ly)) ** 2
        if not clash and not near:
            counter(x0, x1, y0, y1)
            left -= 1
    while left > 0:
        wall = int(rng.integers(4))
        ln, hz = float(rng.uniform(0.3, 1.0)), float(rng.uniform(0.1, 0.3))
        zc = float(rng.uniform(1.4 + hz, 2.3 - hz)) if 2.3 - hz > 1.4 + hz else 1.85
        if wall < 2:
            c = float(rng.uniform(-0.5 * W + 0.5 * ln, 0.5 * W - 0.5 * ln))
            y = (-0.5 * D + 0.025) if wall == 0 else (0.5 * D - 0.025)
            env.static((c, y, zc), (0.5 * ln, 0.025, hz))
        else:
            c = float(rng.uniform(-0.5 * D + 0.5 * ln, 0.5 * D - 0.5 * ln))
            x = (-0.5 * W + 0.025) if wall == 2 else (0.5 * W - 0.025)
            env.static((x, c, zc), (0.025, 0.5 * ln, hz))
        left -= 1
    # floor region: free cells of the room floor outside furniture footprints are
    # handled by placing on a floor "surface" and rejecting furniture overlap
    _add_robot(env, rng, (rb[0], rb[1], 0.12), mobile_base=True)
    floor = _Surfaces()
    floor.add(-0.5 * W + 0.05, 0.5 * W - 0.05, -0.5 * D + 0.05, 0.5 * D - 0.05, 0.0)
    n_surf = len(surf.rects)
    placed = 0
    guard = 0
    while placed < n_obj:
        guard += 1
        if guard > 500 * (n_obj + 1):
            raise RuntimeError("object placement failed")
        shape, dims, m, rho, hz = _random_object(rng, kinds, size_lo, size_hi, mass_fn)
        spot = None
        if n_surf and rng.uniform() < 0.75:
            spot = surf.place(rng, int(rng.integers(n_surf)), rho, keep)
        if spot is None:
            cand = floor.place(rng, 0, rho, keep)
            if cand is not None:
                x, y, _ = cand
                if any(x - rho < f1 and f0 < x + rho and y - rho < g1 and g0 < y + rho
                       for f0, f1, g0, g1 in foot):
                    floor.placed[0].pop()
                    cand = None
            spot = cand
        if spot is None:
            continue
        x, y, z = spot
        q = Q_ID if shape == SPHERE else _yaw_quat(float(rng.uniform(0, 2 * np.pi)))
        env.body(shape, dims, m, (x, y, z + hz), q)
        placed += 1
    return env


def make_config(idx: int, num_envs: int | None = None, seed: int = 0, env_start: int = 0):
    """Scene and solver parameters of benchmark configuration `idx` (1..5).

    1: 64 envs, 8 falling spheres, plane + 4 yawed static boxes, 1x10.
    2: 1024 envs, fixed-base 7-DoF arm + 2 fingers, 12 boxes/capsules on a
       counter of 6 static boxes, 4x20.
    3: 4096 envs, apartment rooms with U{10..60} static boxes, U{4..48}
       objects and a mobile manipulator (planar base), 4x20.
    4: 512 envs, arm hanging over a table pushing a goal box + 5 more boxes,
       4x16, goal position per env.
    5: 16384 envs, apartment rooms with 50 static boxes, 32 objects
       (spheres, capsules, boxes; log-uniform mass), mobile manipulator, 4x20.
    6: 4096 envs, the apartment rooms of 3 with a cabinet drawer and a fridge
       door (articulated receptacles, passive), U{4..32} objects, 4x20; the
       workload of the 20 Hz control wrapper.
    """
    defaults = {1: 64, 2: 1024, 3: 4096, 4: 512, 5: 16384, 6: 4096}
    E = defaults[idx] if num_envs is None else int(num_envs)
    envs = []
    for e in range(env_start, env_start + E):
        rng = _rng(idx, e, seed)
        if idx == 1:
            envs.append(_cfg1_env(rng))
        elif idx == 2:
            envs.append(_cfg2_env(rng))
        elif idx == 3:
            n_obj = int(rng.integers(4, 49))
            n_st = int(rng.integers(10, 61))
            envs.append(_apartment_env(rng, n_obj, n_st, (SPHERE, CAPSULE, BOX), 0.03, 0.15,
                                       lambda: rng.uniform(0.05, 0.5)))
        elif idx == 4:
            envs.append(_cfg4_env(rng))
        elif idx == 5:
            envs.append(_apartment_env(rng, 32, 50, (SPHERE, CAPSULE, BOX), 0.03, 0.20,
                                       lambda: float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))))
        elif idx == 6:
            n_obj = int(rng.integers(4, 33))
            n_st = int(rng.integers(15, 61))
            envs.append(_apartment_env(rng, n_obj, n_st, (SPHERE, CAPSULE, BOX), 0.03, 0.15,
                                       lambda: rng.uniform(0.05, 0.5), receptacles=True))
        else:
            raise ValueError(idx)
    scene = _pack(f"config{idx}", envs, seed, meta={"config": idx})
    cfg = {
        # capacities: about 1.2-1.6x the largest per-env count seen over the first steps
        1: SolverCfg(dt=0.01, substeps=1, iterations=10, friction=0.5, max_contacts=64, max_pairs=64),
        2: SolverCfg(dt=0.01, substeps=4, iterations=20, max_contacts=112, max_pairs=48),
        3: SolverCfg(dt=0.01, substeps=4, iterations=20, max_contacts=160, max_pairs=96),
        4: SolverCfg(dt=0.01, substeps=4, iterations=16, max_contacts=48, max_pairs=24),
        5: SolverCfg(dt=0.01, substeps=4, iterations=20, max_contacts=128, max_pairs=64),
        6: SolverCfg(dt=0.01, substeps=4, iterations=20, max_contacts=160, max_pairs=96),
    }[idx]
    steps = {1: 100, 2: 200, 3: 500, 4: 64, 5: 500, 6: 500}[idx]
    scene.meta["steps"] = steps
    return scene, cfg
