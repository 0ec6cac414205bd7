"""ctypes declarations of the C ABI in include/msh.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

MSH_OK = 0
MSH_ERR_INVALID_ARG = -1
MSH_ERR_CUDA = -2
MSH_ERR_OOM = -3
MSH_ERR_TIMEOUT = -4
MSH_ERR_UNSUPPORTED = -5
EXEC_PLAIN, EXEC_FUSED, EXEC_SUBSTEP = 0, 1, 2

EXPORTS = ("msh_create", "msh_destroy", "msh_last_error", "msh_set_exec", "msh_step", "msh_step_host",
           "msh_detect", "msh_get_status", "msh_clear_status", "msh_scratch_bytes", "msh_workspace_bytes",
           "msh_launches_per_step", "msh_step_static_scratch", "msh_set_tape", "msh_tape_reset",
           "msh_tape_count", "msh_backward", "msh_set_report", "msh_label_events", "msh_set_cameras",
           "msh_render_depth", "msh_set_controller", "msh_control_step",
           "msh_tape_record", "msh_tape_rows", "msh_tape_lambdas")
TASK_PICK, TASK_PLACE, TASK_OPEN, TASK_CLOSE = 0, 1, 2, 3


class SceneDesc(C.Structure):
    _fields_ = [("num_envs", C.c_int32), ("body_off", C.c_void_p), ("static_off", C.c_void_p),
                ("joint_off", C.c_void_p), ("max_dof", C.c_int32), ("body_shape", C.c_void_p),
                ("body_dims", C.c_void_p), ("body_mass", C.c_void_p), ("static_pose", C.c_void_p),
                ("static_half", C.c_void_p), ("joint_type", C.c_void_p), ("joint_parent", C.c_void_p),
                ("joint_child", C.c_void_p), ("joint_dof", C.c_void_p), ("joint_frame_a", C.c_void_p),
                ("joint_frame_b", C.c_void_p), ("joint_gains", C.c_void_p), ("joint_limits", C.c_void_p)]


class SolverCfg(C.Structure):
    _fields_ = [("dt", C.c_float), ("substeps", C.c_int32), ("iterations", C.c_int32), ("mode", C.c_int32),
                ("gravity", C.c_float * 3), ("friction", C.c_float), ("restitution", C.c_float),
                ("contact_offset", C.c_float), ("baumgarte", C.c_float), ("joint_baumgarte", C.c_float),
                ("slop", C.c_float), ("max_contacts", C.c_int32), ("max_pairs", C.c_int32)]


class ReportDesc(C.Structure):
    _fields_ = [("body_flags", C.c_void_p), ("fingers", C.c_void_p), ("target", C.c_void_p),
                ("grasp_min_force", C.c_float), ("grasp_max_angle_deg", C.c_float),
                ("body_force", C.c_void_p), ("target_force", C.c_void_p), ("finger_force", C.c_void_p),
                ("robot_force", C.c_void_p), ("grasped", C.c_void_p)]


class CameraDesc(C.Structure):
    _fields_ = [("num_cameras", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("fov_y", C.c_float),
                ("near_", C.c_float), ("far_", C.c_float), ("body", C.c_void_p), ("pose", C.c_void_p)]


class ControllerDesc(C.Structure):
    _fields_ = [("action_dim", C.c_int32), ("steps_per_action", C.c_int32), ("yaw_dof", C.c_int32),
                ("kind", C.c_void_p), ("action_col", C.c_void_p), ("scale", C.c_void_p), ("lo", C.c_void_p),
                ("hi", C.c_void_p)]


class TrajBatch(C.Structure):
    _fields_ = [("num_traj", C.c_int32), ("num_steps", C.c_int32), ("force", C.c_void_p), ("cumcol", C.c_void_p),
                ("dist", C.c_void_p), ("artq", C.c_void_p), ("flags", C.c_void_p), ("length", C.c_void_p),
                ("art_range", C.c_void_p), ("art_fridge", C.c_void_p), ("collision_limit", C.c_float),
                ("goal_radius", C.c_float)]


class State(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("quat", C.c_void_p), ("linvel", C.c_void_p), ("angvel", C.c_void_p)]


_lib = None


def load(build_if_missing: bool = True):
    """Loads libmsh.so; raises if it is missing and cannot be built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmsh.so not found at {path}; run paper_2412_13211_b300.build.build()")
    lib = C.CDLL(path)
    P, I32, F = C.c_void_p, C.c_int32, C.c_float
    lib.msh_create.argtypes = [P, P, P]
    lib.msh_destroy.argtypes = [P]
    lib.msh_destroy.restype = None
    lib.msh_last_error.restype = C.c_char_p
    lib.msh_set_exec.argtypes = [P, I32, I32, I32]
    lib.msh_step.argtypes = [P, P, P, F, I32, P]
    lib.msh_step_host.argtypes = [P, P, P, P, P, P, F, I32, P]
    lib.msh_step_static_scratch.argtypes = [P, P, P, F, I32, P]
    lib.msh_set_tape.argtypes = [P, I32]
    lib.msh_set_report.argtypes = [P, P]
    lib.msh_set_cameras.argtypes = [P, P]
    lib.msh_render_depth.argtypes = [P, P, P, P]
    lib.msh_set_controller.argtypes = [P, P]
    lib.msh_control_step.argtypes = [P, P, P, P, P]
    lib.msh_label_events.argtypes = [I32, P, I32, P, P, P, P]
    lib.msh_tape_reset.argtypes = [P]
    lib.msh_tape_record.argtypes = [P, I32]
    lib.msh_tape_count.argtypes = [P]
    lib.msh_tape_count.restype = C.c_int32
    lib.msh_tape_rows.argtypes = [P]
    lib.msh_tape_rows.restype = C.c_int32
    lib.msh_tape_lambdas.argtypes = [P, I32, P, P]
    lib.msh_backward.argtypes = [P, P, P, P, P, P]
    lib.msh_detect.argtypes = [P] * 12 + [P]
    lib.msh_get_status.argtypes = [P, P, P]
    lib.msh_clear_status.argtypes = [P, P]
    lib.msh_scratch_bytes.argtypes = [P]
    lib.msh_scratch_bytes.restype = C.c_int64
    lib.msh_workspace_bytes.argtypes = [P]
    lib.msh_workspace_bytes.restype = C.c_int64
    lib.msh_launches_per_step.argtypes = [P]
    lib.msh_launches_per_step.restype = C.c_int32
    for name in EXPORTS:
        getattr(lib, name)
        if name not in ("msh_destroy", "msh_last_error", "msh_scratch_bytes", "msh_workspace_bytes",
                        "msh_launches_per_step", "msh_tape_count", "msh_tape_rows"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(rc: int, what: str):
    if rc != MSH_OK:
        msg = load().msh_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed ({rc}): {msg}")
