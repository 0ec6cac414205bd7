"""Oracle of the control wrapper (test infrastructure only: the tests, the
smoke check and the benchmark's CPU legs use it; the product never does).

The paper's environments take one normalised action per control step and run
several physics steps under it: Sec. 4.1 names a PD joint delta-position
controller for the arm, linear and angular velocity for the base and an
action space normalised to [-1, 1]; Sec. 4.2 runs the physics at 100 Hz under
20 Hz control, i.e. five physics steps per action. The paper does not spell
out the controllers' arithmetic; this module fixes these readings:

  K1  each action component is first clipped to [-1, 1]; a NaN component
      counts as -1 (IEEE fmax/fmin drop a NaN operand);
  K2  delta position: the new target is the previous TARGET plus the clipped
      action times the column's delta, then clipped to the DoF's range;
  K3  gripper: absolute, target = lo + (a + 1) / 2 * (hi - lo), both fingers
      from one action column;
  K4  base: v = a_v * speed and w = a_w * turn act over the control period
      dt_c = steps * dt with the yaw TARGET from before the update:
      x += v cos(yaw) dt_c, y += v sin(yaw) dt_c, yaw += w dt_c, each then
      clipped to its range;
  K5  columns of passive joints keep their targets;
  K6  one control step is the controller followed by `steps` physics steps
      that all use the new targets.

In FP32 every operation rounds to FP32 in the order written here (the
products scale * a, then * cos(yaw), then * dt_c; the gripper's
((a + 1) * 0.5) * (hi - lo) + lo); cos and sin of the FP32 yaw are taken in
FP64 and rounded once.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o

HOLD, DELTA, ABS, BASE_X, BASE_Y, BASE_YAW = 0, 1, 2, 3, 4, 5


def control_dt(steps: int, dt: float, precision: str = "f32"):
    """dt_c = steps * dt (FP32: both operands and the product in FP32)."""
    if precision == "f32":
        return np.float32(np.float32(steps) * np.float32(dt))
    return float(steps) * float(dt)


def controller(spec, action, targets, dt_c, precision: str = "f32"):
    """One application of the controller to every env (K1-K5).

    action [E, A] and targets [E, max_dof]; returns the new targets."""
    T = np.float32 if precision == "f32" else np.float64
    a_all = np.asarray(action).astype(T)
    t_old = np.asarray(targets).astype(T)
    out = t_old.copy()
    dt_c = T(dt_c)
    one, half = T(1.0), T(0.5)
    E, D = out.shape
    for e in range(E):
        yaw0 = t_old[e, spec.yaw_dof] if spec.yaw_dof >= 0 else T(0.0)
        c, s = T(np.cos(np.float64(yaw0))), T(np.sin(np.float64(yaw0)))
        for d in range(D):
            k = int(spec.kind[d])
            if k == HOLD:
                continue
            a = np.fmin(np.fmax(a_all[e, int(spec.action[d])], -one), one)          # K1
            lo, hi, sc = T(spec.lo[d]), T(spec.hi[d]), T(spec.scale[d])
            t = t_old[e, d]
            if k == DELTA:                                                           # K2
                t = t + a * sc
            elif k == ABS:                                                           # K3
                t = (a + one) * half * (hi - lo) + lo
            elif k == BASE_X:                                                        # K4
                t = t + a * sc * c * dt_c
            elif k == BASE_Y:
                t = t + a * sc * s * dt_c
            elif k == BASE_YAW:
                t = t + a * sc * dt_c
            else:
                raise ValueError(f"controller kind {k}")
            out[e, d] = np.fmin(np.fmax(t, lo), hi)
    return out


def control_step(scene, cfg, spec, state, action, targets, precision: str = "f32", threads: int = 0):
    """One control step (K6): returns (state, targets, status)."""
    dt_c = control_dt(spec.steps_per_action, cfg.dt, precision)
    new = controller(spec, action, targets, dt_c, precision)
    tg = np.repeat(np.asarray(new, np.float32)[None], spec.steps_per_action, axis=0)   # drives read FP32 targets
    st, status = _o.step(scene, cfg, state, tg, spec.steps_per_action, precision, threads)
    return st, new, status


def rollout(scene, cfg, spec, state, actions, targets, precision: str = "f32", threads: int = 0):
    """len(actions) control steps from (state, targets)."""
    status = None
    for a in actions:
        state, targets, s = control_step(scene, cfg, spec, state, a, targets, precision, threads)
        status = s if status is None else status | s
    return state, targets, status
