"""Tiny hand-built scenes for closed-form and invariant tests."""
import numpy as np

from paper_2412_13211_b300 import scenes as S


def scene_from_envs(envs, name="unit"):
    return S._pack(name, envs, 0)


def env():
    return S._Env()


def cfg(**kw):
    c = S.SolverCfg()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def quat_mul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def quat_rotate(q, v):
    qv = quat_mul(quat_mul(q, [0.0, *v]), [q[0], -q[1], -q[2], -q[3]])
    return qv[1:]


def axis_angle(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return (float(np.cos(ang / 2)),) + tuple(float(v) for v in np.sin(ang / 2) * axis)
