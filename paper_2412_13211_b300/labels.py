"""Event labeling and trajectory categorization on the GPU (msh_label_events).

Takes the per-step records of a batch of trajectories of one subtask as CUDA
tensors, step-major [T, N] (see trajectories.py for the layout), and returns
each trajectory's event count, first events and success/failure mode
(Appendix A.5). Argument marshalling only: the scan runs in the library.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import TrajBatch, check

PICK, PLACE, OPEN, CLOSE = _lib.TASK_PICK, _lib.TASK_PLACE, _lib.TASK_OPEN, _lib.TASK_CLOSE
EVENTS = {
    PICK: ("contact", "grasped", "dropped", "success", "excessive_collisions"),
    PLACE: ("grasped", "obj_at_goal", "released_at_goal", "released_outside_goal", "obj_left_goal", "success",
            "excessive_collisions"),
    OPEN: ("contact", "opened", "slightly_opened", "closed", "success", "excessive_collisions"),
    CLOSE: ("contact", "closed", "slightly_closed", "opened", "success", "excessive_collisions"),
}


def _p(t):
    return t.data_ptr() if t is not None else None


def label_events(task: int, traj: dict, max_events: int = 32, collision_limit: float = 0.0,
                 goal_radius: float = 0.0, stream=None):
    """traj: CUDA tensors cumcol/force/dist/artq [T, N] float32, flags [T, N]
    uint8, optional length [N] int32, art_range [N, 2] float32, art_fridge [N]
    uint8. Returns (events int8 [N, max_events], num_events int32 [N],
    label int32 [N]) on the same device."""
    lib = _lib.load()
    cum = traj["cumcol"]
    T, N = cum.shape
    dev = cum.device
    keep = {k: (v.contiguous() if v is not None else None) for k, v in traj.items()}
    b = TrajBatch()
    b.num_traj, b.num_steps = N, T
    for k in ("force", "cumcol", "dist", "artq", "flags", "length", "art_range", "art_fridge"):
        setattr(b, k, _p(keep.get(k)))
    b.collision_limit, b.goal_radius = float(collision_limit), float(goal_radius)
    events = torch.empty((N, max_events), dtype=torch.int8, device=dev)
    num = torch.empty(N, dtype=torch.int32, device=dev)
    lab = torch.empty(N, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        check(lib.msh_label_events(int(task), C.byref(b), int(max_events), C.c_void_p(events.data_ptr()),
                                   C.c_void_p(num.data_ptr()), C.c_void_p(lab.data_ptr()),
                                   C.c_void_p(s.cuda_stream)), "msh_label_events")
    return events, num, lab


def to_device(traj: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(v).to(device) for k, v in traj.items()}
