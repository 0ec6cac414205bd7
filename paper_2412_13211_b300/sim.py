"""Thin PyTorch front end of the C ABI: device memory and streams only.

Every stage of the step runs in libmsh.so; this module marshals arrays into
the descriptor structs and passes tensor data pointers and the current CUDA
stream. There is no CPU fallback: constructing a simulator without a CUDA
device or without the library raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import EXEC_FUSED, EXEC_PLAIN, EXEC_SUBSTEP, CameraDesc, ControllerDesc, ReportDesc, SceneDesc, SolverCfg, State, check


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def make_desc(scene):
    """Scene descriptor struct plus the host arrays it points to (keep both alive)."""
    keep = dict(
        body_off=_c(scene.body_off, np.int32), static_off=_c(scene.static_off, np.int32),
        joint_off=_c(scene.joint_off, np.int32), body_shape=_c(scene.body_shape, np.int32),
        body_dims=_c(scene.body_dims, np.float32), body_mass=_c(scene.body_mass, np.float32),
        static_pose=_c(scene.static_pose, np.float32), static_half=_c(scene.static_half, np.float32),
        joint_type=_c(scene.joint_type, np.int32), joint_parent=_c(scene.joint_parent, np.int32),
        joint_child=_c(scene.joint_child, np.int32), joint_dof=_c(scene.joint_dof, np.int32),
        joint_frame_a=_c(scene.joint_frame_a, np.float32), joint_frame_b=_c(scene.joint_frame_b, np.float32),
        joint_gains=_c(scene.joint_gains, np.float32), joint_limits=_c(scene.joint_limits, np.float32))
    d = SceneDesc()
    d.num_envs = scene.num_envs
    d.max_dof = scene.max_dof
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data if v.size else None)
    return d, keep


def make_cfg(cfg) -> SolverCfg:
    c = SolverCfg()
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


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class MshSim:
    """A batch of environments resident on one GPU.

    state: pos [B,3], quat [B,4], linvel [B,3], angvel [B,3] float32 CUDA
    tensors, updated in place by `step`."""

    def __init__(self, scene, cfg, device="cuda", exec_form: str = "fused", threads_per_env: int = 0,
                 use_graph: bool = False):
        if not torch.cuda.is_available():
            raise RuntimeError("MshSim needs a CUDA device; the step has no CPU implementation")
        self.lib = _lib.load()
        self.scene, self.cfg = scene, cfg
        self.tape_owner = None   # the rollout whose forward pass recorded the tape (see autograd.rollout)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            desc, keep = make_desc(scene)
            self._cfg = make_cfg(cfg)
            h = C.c_void_p()
            check(self.lib.msh_create(C.byref(desc), C.byref(self._cfg), C.byref(h)), "msh_create")
            self.handle = h
        del keep
        dev = self.device
        self.pos = torch.from_numpy(_c(scene.pos, np.float32)).to(dev)
        self.quat = torch.from_numpy(_c(scene.quat, np.float32)).to(dev)
        self.linvel = torch.from_numpy(_c(scene.linvel, np.float32)).to(dev)
        self.angvel = torch.from_numpy(_c(scene.angvel, np.float32)).to(dev)
        self.max_dof = scene.max_dof
        self.targets = torch.zeros((scene.num_envs, max(scene.max_dof, 1)), dtype=torch.float32, device=dev)
        self.set_exec(exec_form, threads_per_env, use_graph)

    # -- configuration ------------------------------------------------------
    def set_exec(self, exec_form: str = "fused", threads_per_env: int = 0, use_graph: bool = False):
        """exec_form: "fused" (one persistent launch per step), "substep" (one launch
        per substep) or "plain" (one launch per stage); threads_per_env 0 = default."""
        form = {"plain": EXEC_PLAIN, "fused": EXEC_FUSED, "substep": EXEC_SUBSTEP}[exec_form]
        with torch.cuda.device(self.device):
            check(self.lib.msh_set_exec(self.handle, form, int(threads_per_env), int(bool(use_graph))),
                  "msh_set_exec")
        self.exec_form, self.threads_per_env, self.use_graph = exec_form, threads_per_env, use_graph

    @property
    def launches_per_step(self) -> int:
        return int(self.lib.msh_launches_per_step(self.handle))

    @property
    def scratch_bytes(self) -> int:
        return int(self.lib.msh_scratch_bytes(self.handle))

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.msh_workspace_bytes(self.handle))

    # -- state ----------------------------------------------------------------
    def _state(self):
        st = State()
        st.pos, st.quat = self.pos.data_ptr(), self.quat.data_ptr()
        st.linvel, st.angvel = self.linvel.data_ptr(), self.angvel.data_ptr()
        return st

    def set_state(self, pos, quat, linvel, angvel):
        for dst, src in ((self.pos, pos), (self.quat, quat), (self.linvel, linvel), (self.angvel, angvel)):
            dst.copy_(torch.as_tensor(np.asarray(src, np.float32)).to(self.device))

    def state_numpy(self):
        torch.cuda.synchronize(self.device)
        return tuple(t.detach().cpu().numpy().copy() for t in (self.pos, self.quat, self.linvel, self.angvel))

    # -- stepping -------------------------------------------------------------
    def step(self, targets=None, dt: float = 0.0, substeps: int = 0, stream=None):
        """One step of every env; `targets` [E, max_dof] CUDA tensor or array (absolute PD targets)."""
        if targets is not None and self.max_dof > 0:
            if not (isinstance(targets, torch.Tensor) and targets.is_cuda and targets.dtype == torch.float32
                    and targets.is_contiguous()):
                self.targets.copy_(torch.as_tensor(np.asarray(targets, np.float32)).reshape(self.targets.shape))
                targets = self.targets
        else:
            targets = self.targets
        st = self._state()
        with torch.cuda.device(self.device):
            check(self.lib.msh_step(self.handle, C.byref(st), _ptr(targets), float(dt), int(substeps),
                                    _stream(stream)), "msh_step")

    def step_host(self, pos, quat, linvel, angvel, targets, dt: float = 0.0, substeps: int = 0, stream=None):
        """Step with HOST arrays (pinned tensors or contiguous numpy); copies in and out."""
        def hp(a):
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.is_contiguous() and a.dtype == torch.float32
                return C.c_void_p(a.data_ptr())
            assert a.dtype == np.float32 and a.flags.c_contiguous
            return a.ctypes.data_as(C.c_void_p)
        with torch.cuda.device(self.device):
            check(self.lib.msh_step_host(self.handle, hp(pos), hp(quat), hp(linvel), hp(angvel),
                                         hp(targets) if targets is not None else None, float(dt), int(substeps),
                                         _stream(stream)), "msh_step_host")

    def detect(self, stream=None):
        """Collision stage at the current poses: AABBs, pairs, contacts, colours (numpy)."""
        sc, cfg = self.scene, self.cfg
        E, P, K = sc.num_envs, cfg.max_pairs, cfg.max_contacts
        dev = self.device
        out = dict(
            aabb_body=torch.zeros((max(sc.num_bodies, 1), 6), device=dev),
            aabb_static=torch.zeros((max(sc.num_statics, 1), 6), device=dev),
            pair_count=torch.zeros(E, dtype=torch.int32, device=dev),
            pairs=torch.full((E, P, 2), -1, dtype=torch.int32, device=dev),
            contact_count=torch.zeros(E, dtype=torch.int32, device=dev),
            contact_ids=torch.full((E, K, 2), -1, dtype=torch.int32, device=dev),
            contact_geom=torch.zeros((E, K, 10), device=dev),
            manifold_count=torch.zeros(E, dtype=torch.int32, device=dev),
            colours=torch.full((sc.num_joints + E * P,), -1, dtype=torch.int32, device=dev),
            ncolours=torch.zeros(E, dtype=torch.int32, device=dev))
        st = self._state()
        with torch.cuda.device(dev):
            check(self.lib.msh_detect(self.handle, C.byref(st), *[_ptr(out[k]) for k in (
                "aabb_body", "aabb_static", "pair_count", "pairs", "contact_count", "contact_ids",
                "contact_geom", "manifold_count", "colours", "ncolours")], _stream(stream)), "msh_detect")
            torch.cuda.synchronize(dev)
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["aabb_body"] = res["aabb_body"][:sc.num_bodies]
        res["aabb_static"] = res["aabb_static"][:sc.num_statics]
        return res

    # -- control wrapper --------------------------------------------------------
    def set_controller(self, spec):
        """Controller of the control steps (msh_set_controller) from a
        scenes.ControllerSpec; makes `self.ctrl_targets` [E, max_dof], the
        PD targets the controller updates, start at the scene's targets0."""
        D = self.max_dof
        kind = np.ascontiguousarray(spec.kind, np.int32).reshape(D)
        col = np.ascontiguousarray(np.where(spec.kind == 0, 0, spec.action), np.int32).reshape(D)
        scale = np.ascontiguousarray(spec.scale, np.float32).reshape(D)
        lo = np.ascontiguousarray(spec.lo, np.float32).reshape(D)
        hi = np.ascontiguousarray(spec.hi, np.float32).reshape(D)
        d = ControllerDesc(int(spec.action_dim), int(spec.steps_per_action), int(spec.yaw_dof), kind.ctypes.data,
                           col.ctypes.data, scale.ctypes.data, lo.ctypes.data, hi.ctypes.data)
        with torch.cuda.device(self.device):
            check(self.lib.msh_set_controller(self.handle, C.byref(d)), "msh_set_controller")
        self.ctrl_spec = spec
        self.ctrl_targets = torch.as_tensor(np.asarray(self.scene.targets0, np.float32)).to(self.device).contiguous()
        self.ctrl_action = torch.zeros((self.scene.num_envs, int(spec.action_dim)), dtype=torch.float32,
                                       device=self.device)

    def control_step(self, action=None, targets=None, stream=None):
        """One control step (msh_control_step): the controller turns `action`
        [E, action_dim] into new PD targets (in place in `targets`, default
        self.ctrl_targets), then the physics steps run. A CUDA float32
        contiguous `action` is used as is; anything else is copied into a
        buffer owned by this object first."""
        if action is not None:
            if not (isinstance(action, torch.Tensor) and action.is_cuda and action.dtype == torch.float32
                    and action.is_contiguous()):
                self.ctrl_action.copy_(torch.as_tensor(np.asarray(action, np.float32)).reshape(self.ctrl_action.shape))
                action = self.ctrl_action
        else:
            action = self.ctrl_action
        if targets is None:
            targets = self.ctrl_targets
        assert targets.is_cuda and targets.dtype == torch.float32 and targets.is_contiguous()
        st = self._state()
        with torch.cuda.device(self.device):
            check(self.lib.msh_control_step(self.handle, C.byref(st), _ptr(action), _ptr(targets), _stream(stream)),
                  "msh_control_step")
        return targets

    # -- depth cameras ---------------------------------------------------------
    def set_cameras(self, body, pose, width: int = 128, height: int = 128, fov_y: float = np.pi / 2,
                    near: float = 0.01, far: float = 10.0):
        """Depth cameras (msh_set_cameras): body [E, ncam] env-local mount bodies
        (-1: world), pose [E, ncam, 7] mount-local poses (position, quaternion)."""
        E = self.scene.num_envs
        b = np.ascontiguousarray(body, np.int32).reshape(E, -1)
        ps = np.ascontiguousarray(pose, np.float32).reshape(E, b.shape[1], 7)
        d = CameraDesc(b.shape[1], int(width), int(height), float(fov_y), float(near), float(far),
                       b.ctypes.data, ps.ctypes.data)
        with torch.cuda.device(self.device):
            check(self.lib.msh_set_cameras(self.handle, C.byref(d)), "msh_set_cameras")
        self.cam_shape = (E, b.shape[1], int(height), int(width))

    def render_depth(self, out=None, stream=None):
        """Depth images [E, ncam, H, W] (z-depth in m, 0 = no hit) at the current state."""
        if out is None:
            out = torch.empty(self.cam_shape, dtype=torch.float32, device=self.device)
        st = self._state()
        with torch.cuda.device(self.device):
            check(self.lib.msh_render_depth(self.handle, C.byref(st), C.c_void_p(out.data_ptr()), _stream(stream)),
                  "msh_render_depth")
        return out

    # -- contact report ---------------------------------------------------------
    def set_report(self, body_flags, fingers=None, target=None, grasp_min_force: float = 0.5,
                   grasp_max_angle_deg: float = 85.0):
        """Turns on the per-step contact report (msh_set_report) into device
        tensors owned by this object: body_force [B,3], target_force [E,3],
        finger_force [E,2,3], robot_force [E] (accumulated; zero it with
        reset_robot_force) and grasped [E]. body_flags [B]: bit 0 robot link,
        bit 1 end-effector link; fingers [E,2] and target [E] are env-local
        body ids (-1: none). Returns the dict of output tensors."""
        sc, dev = self.scene, self.device
        E, B = sc.num_envs, sc.num_bodies
        out = dict(body_force=torch.zeros((max(B, 1), 3), device=dev), target_force=torch.zeros((E, 3), device=dev),
                   finger_force=torch.zeros((E, 2, 3), device=dev), robot_force=torch.zeros(E, device=dev),
                   grasped=torch.zeros(E, dtype=torch.int32, device=dev))
        flags = np.ascontiguousarray(body_flags, np.int32).reshape(B)
        fing = None if fingers is None else np.ascontiguousarray(fingers, np.int32).reshape(E, 2)
        tgt = None if target is None else np.ascontiguousarray(target, np.int32).reshape(E)
        d = ReportDesc()
        d.body_flags = flags.ctypes.data
        d.fingers = fing.ctypes.data if fing is not None else None
        d.target = tgt.ctypes.data if tgt is not None else None
        d.grasp_min_force, d.grasp_max_angle_deg = float(grasp_min_force), float(grasp_max_angle_deg)
        for k in ("body_force", "target_force", "finger_force", "robot_force", "grasped"):
            setattr(d, k, out[k].data_ptr())
        with torch.cuda.device(dev):
            check(self.lib.msh_set_report(self.handle, C.byref(d)), "msh_set_report")
        self.report_out = out
        return out

    def clear_report(self):
        with torch.cuda.device(self.device):
            check(self.lib.msh_set_report(self.handle, None), "msh_set_report")
        self.report_out = None

    def reset_robot_force(self):
        if getattr(self, "report_out", None) is not None:
            self.report_out["robot_force"].zero_()

    def report(self) -> dict:
        """numpy copies of the report outputs (synchronises)."""
        res = {k: v.cpu().numpy() for k, v in self.report_out.items()}
        res["body_force"] = res["body_force"][:self.scene.num_bodies]
        return res

    # -- adjoint --------------------------------------------------------------
    def set_tape(self, max_steps: int):
        """max_steps > 0: record the next steps (room for max_steps); 0: stop
        recording (memory kept); -1: stop and free the tape."""
        self.tape_owner = None
        with torch.cuda.device(self.device):
            check(self.lib.msh_set_tape(self.handle, int(max_steps)), "msh_set_tape")

    def tape_reset(self):
        self.tape_owner = None
        check(self.lib.msh_tape_reset(self.handle), "msh_tape_reset")

    def tape_record(self, on: bool):
        """Pauses (False) or resumes (True) recording, keeping the recorded steps."""
        check(self.lib.msh_tape_record(self.handle, int(bool(on))), "msh_tape_record")

    @property
    def tape_count(self) -> int:
        return int(self.lib.msh_tape_count(self.handle))

    def backward(self, adj_out, adj_targets=None, adj_mass=None, stream=None):
        """Reverses the last recorded step. adj_out: adjoints (pos, quat, linvel,
        angvel) of the state after it; returns the adjoints of the state before
        it. adj_targets [E, max_dof] receives that step's target adjoint;
        adj_mass [B] accumulates."""
        def st(ts):
            x = State()
            x.pos, x.quat, x.linvel, x.angvel = (t.data_ptr() for t in ts)
            return x
        ins = [t.contiguous() for t in adj_out]
        outs = [torch.empty_like(t) for t in ins]
        a, b = st(ins), st(outs)
        with torch.cuda.device(self.device):
            check(self.lib.msh_backward(self.handle, C.byref(a), C.byref(b), _ptr(adj_targets), _ptr(adj_mass),
                                        _stream(stream)), "msh_backward")
        return tuple(outs)

    def tape_lambdas(self, slot: int = 0, stream=None) -> np.ndarray:
        """Impulses after every sweep of recorded step `slot`:
        [E, substeps, iterations, rows] (see msh_tape_lambdas for the rows)."""
        rows = int(self.lib.msh_tape_rows(self.handle))
        out = np.zeros((self.scene.num_envs, self.cfg.substeps, self.cfg.iterations, rows), np.float32)
        with torch.cuda.device(self.device):
            check(self.lib.msh_tape_lambdas(self.handle, int(slot), out.ctypes.data_as(C.c_void_p), _stream(stream)),
                  "msh_tape_lambdas")
        return out

    def status(self, stream=None) -> np.ndarray:
        out = np.zeros(self.scene.num_envs, np.int32)
        with torch.cuda.device(self.device):
            check(self.lib.msh_get_status(self.handle, out.ctypes.data_as(C.c_void_p), _stream(stream)),
                  "msh_get_status")
        return out

    def clear_status(self, stream=None):
        with torch.cuda.device(self.device):
            check(self.lib.msh_clear_status(self.handle, _stream(stream)), "msh_clear_status")

    def close(self):
        if getattr(self, "handle", None):
            with torch.cuda.device(self.device):
                self.lib.msh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
