"""Pins of the depth-camera oracle (the paper's per-env RGB-D cameras,
Sec. 4.2, restated as ray casting against the env's primitives).

Closed forms: a camera looking straight down at the ground sees its height
at every pixel; a box face seen head-on has one z-depth; a sphere's silhouette
is the cone of half-angle asin(r/d); a capsule seen side-on is nearest along
its axis. Independently of the oracle's closed forms, random scenes are
ray-marched on signed distance functions (sphere tracing) in FP64.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, env, scene_from_envs

W = H = 32
FOV = np.pi / 2
FOCAL = float(np.float32((H / 2) / np.tan(FOV / 2)))
NEAR, FAR = 0.01, 10.0


def _render(sc, cam_pose, cam_body=None, precision="f64", W_=W, H_=H, focal=FOCAL):
    E = sc.num_envs
    cam_pose = np.asarray(cam_pose, np.float64).reshape(E, -1, 7)
    body = np.full(cam_pose.shape[:2], -1, np.int32) if cam_body is None else np.asarray(cam_body, np.int32)
    return oracle.render_depth(sc, sc.pos, sc.quat, body, cam_pose, W_, H_, focal, NEAR, FAR, precision)


def _rays(focal=FOCAL, W_=W, H_=H):
    """Camera-frame pixel rays (1, -(u - W/2)/f, -(v - H/2)/f)."""
    col, row = np.meshgrid(np.arange(W_) + 0.5, np.arange(H_) + 0.5)
    return np.stack([np.ones_like(col), -(col - W_ / 2) / focal, -(row - H_ / 2) / focal], -1)


def _empty():
    e = env()
    e.body(S.SPHERE, (0.01,), 1.0, (50.0, 50.0, 50.0))     # far away, out of view
    return e


def test_ground_seen_from_above_is_flat():
    sc = scene_from_envs([_empty()])
    q = axis_angle((0.0, 1.0, 0.0), np.pi / 2)                  # +x turned to -z
    d = _render(sc, [(0.25, -0.5, 1.5) + tuple(q)])
    np.testing.assert_allclose(d[0, 0], 1.5, rtol=0, atol=1e-6)   # the quaternion is rounded to f32


def test_box_face_head_on_has_one_depth():
    e = _empty()
    e.static((2.25, 0.0, 1.0), (0.25, 0.5, 0.5))               # face at x = 2.0 (exact in f32)
    sc = scene_from_envs([e])
    d = _render(sc, [(0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0)])[0, 0]
    r = _rays()
    y, z = 2.0 * r[..., 1], 1.0 + 2.0 * r[..., 2]               # where each ray crosses the face plane
    inside = (np.abs(y) < 0.5 - 1e-9) & (np.abs(z - 1.0) < 0.5 - 1e-9)
    assert inside.sum() > 50
    np.testing.assert_allclose(d[inside], 2.0, rtol=0, atol=1e-12)
    assert (d[~inside] != 2.0).all()


def test_sphere_silhouette_is_a_cone():
    e = env()
    e.body(S.SPHERE, (0.5,), 1.0, (3.0, 0.0, 2.0))
    sc = scene_from_envs([e])
    d = _render(sc, [(0.0, 0.0, 2.0, 1.0, 0.0, 0.0, 0.0)])[0, 0]
    r = _rays()
    ang = np.arccos(r[..., 0] / np.linalg.norm(r, axis=-1))
    half = np.arcsin(0.5 / 3.0)
    hit_in = ang < half - 1e-6
    miss_out = ang > half + 1e-6
    assert hit_in.sum() > 10
    assert (d[hit_in] > 0).all() and (d[hit_in] < 3.0).all()
    # outside the cone the rays see the ground (z-depth 2 / -r_z) or nothing
    rz = r[..., 2]
    ground = np.where(rz < 0, 2.0 / np.where(rz < 0, -rz, 1.0), 0.0)
    ground = np.where(ground <= FAR, ground, 0.0)
    np.testing.assert_allclose(d[miss_out], ground[miss_out], rtol=0, atol=1e-9)
    # the pixel next to the axis (half a pixel off in both directions) sees near the front point
    assert 2.5 < d[H // 2, W // 2] < 2.52


def test_capsule_side_on_nearest_along_its_axis():
    e = env()
    q = axis_angle((0.0, 1.0, 0.0), -np.pi / 2)                 # capsule axis (local x) along world z
    e.body(S.CAPSULE, (0.25, 0.5), 1.0, (2.0, 0.0, 1.0), q)
    sc = scene_from_envs([e])
    d = _render(sc, [(0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0)])[0, 0]
    r = _rays()
    # centre column crosses the axis plane; rows whose ray meets the cylinder side between the caps
    zc = 1.0 + 1.75 * r[:, W // 2, 2]
    rows = np.abs(zc - 1.0) < 0.45
    # seen from above, the ray (s, a s) meets the cylinder's circle (x - 2)^2 + y^2 = 0.25^2 first at
    # (1 + a^2) s^2 - 4 s + (4 - 0.0625) = 0 (a: the column's half-pixel horizontal slope)
    a = r[rows, W // 2, 1]
    A = 1.0 + a * a
    expect = (4.0 - np.sqrt(16.0 - 4.0 * A * (4.0 - 0.0625))) / (2.0 * A)
    # (the capsule's quaternion is stored in f32: its axis leans by ~1e-8)
    np.testing.assert_allclose(d[rows, W // 2], expect, rtol=0, atol=1e-7)


def _sdf(p, prims):
    out = np.full(p.shape[:-1], np.inf)
    for kind, a in prims:
        if kind == "sphere":
            c, r = a
            v = np.linalg.norm(p - c, axis=-1) - r
        elif kind == "box":
            c, R, h = a
            q = np.abs((p - c) @ R) - h
            v = np.linalg.norm(np.maximum(q, 0), axis=-1) + np.minimum(q.max(-1), 0)
        elif kind == "capsule":
            c, R, L, r = a
            ax = R[:, 0]
            t = np.clip((p - c) @ ax, -L, L)
            v = np.linalg.norm(p - (c + t[..., None] * ax), axis=-1) - r
        else:
            v = p[..., 2]
        out = np.minimum(out, v)
    return out


def _qmat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_scenes_against_sphere_tracing(seed):
    rng = np.random.default_rng(seed)
    e = env()
    prims = [("plane", None)]
    for k in range(6):
        c = np.array([rng.uniform(1.5, 4.0), rng.uniform(-1.5, 1.5), rng.uniform(0.3, 1.8)])
        ax = rng.normal(size=3)
        q = axis_angle(ax, rng.uniform(0, np.pi))
        kind = k % 3
        if kind == 0:
            r = rng.uniform(0.1, 0.4)
            e.body(S.SPHERE, (r,), 1.0, tuple(c), q)
        elif kind == 1:
            r, L = rng.uniform(0.05, 0.2), rng.uniform(0.1, 0.4)
            e.body(S.CAPSULE, (r, L), 1.0, tuple(c), q)
        else:
            h = rng.uniform(0.1, 0.4, size=3)
            e.body(S.BOX, tuple(h), 1.0, tuple(c), q)
    e.static((3.0, 2.5, 1.0), (1.0, 0.1, 1.0), tuple(axis_angle((0, 0, 1), 0.3)))
    sc = scene_from_envs([e])
    # the scene as stored (f32), in f64, for the SDFs
    for i in range(sc.num_bodies):
        c = sc.pos[i].astype(np.float64)
        R = _qmat(sc.quat[i].astype(np.float64))
        dm = sc.body_dims[i].astype(np.float64)
        sh = int(sc.body_shape[i])
        prims.append(("sphere", (c, dm[0])) if sh == 0 else ("capsule", (c, R, dm[1], dm[0])) if sh == 1
                     else ("box", (c, R, dm[:3])))
    sp = sc.static_pose[0].astype(np.float64)
    prims.append(("box", (sp[:3], _qmat(sp[3:]), sc.static_half[0].astype(np.float64))))
    cam_q = axis_angle((0.0, 1.0, 0.0), 0.3)                    # pitched down
    cam = np.array([0.0, 0.0, 1.6])
    d = _render(sc, [tuple(cam) + tuple(cam_q)])[0, 0]
    Rc = _qmat(np.array(cam_q, np.float32).astype(np.float64))
    rays = _rays() @ Rc.T
    rows, cols = rng.integers(0, H, 60), rng.integers(0, W, 60)
    checked = 0
    for rr, cc in zip(rows, cols):
        D = rays[rr, cc]
        n = np.linalg.norm(D)
        u = D / n
        t, p = 0.0, cam.astype(np.float64)
        hit = None
        for _ in range(4000):
            v = _sdf(p[None], prims)[0]
            if v < 1e-10:
                hit = t
                break
            t += v
            p = cam + t * u
            if t > FAR * n:
                break
        if hit is None:
            assert d[rr, cc] == 0.0
        else:
            s = hit / n
            if s <= FAR and s >= NEAR:
                assert abs(d[rr, cc] - s) < 1e-6, (rr, cc, d[rr, cc], s)
                checked += 1
    assert checked > 30


def test_mounted_camera_follows_its_body_and_f32_tracks_f64():
    e = env()
    e.body(S.BOX, (0.1, 0.1, 0.1), 1.0, (0.0, 0.0, 1.0), axis_angle((0, 0, 1), 0.7))
    e.static((2.0, 1.5, 0.5), (0.3, 0.3, 0.5))
    e.body(S.SPHERE, (0.3,), 1.0, (1.5, 1.0, 0.6))
    sc = scene_from_envs([e])
    local = (0.2, 0.0, 0.1) + tuple(axis_angle((0, 1, 0), 0.2))
    d_mount = _render(sc, [local], cam_body=[[0]])[0, 0]
    # the same camera given in the world frame
    qb = sc.quat[0].astype(np.float64)
    pw = sc.pos[0].astype(np.float64) + _qmat(qb) @ np.array(local[:3])
    w0, x0, y0, z0 = qb
    w1, x1, y1, z1 = local[3:]
    qw = (w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1, w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
          w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1, w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1)
    d_world = _render(sc, [tuple(pw) + qw])[0, 0]
    np.testing.assert_allclose(d_mount, d_world, rtol=0, atol=2e-6)   # world pose passes through f32
    d32 = _render(sc, [local], cam_body=[[0]], precision="f32")[0, 0]
    both = (d32 > 0) & (d_mount > 0)
    assert both.mean() > 0.5
    assert np.abs(d32[both] - d_mount[both]).max() < 1e-4
