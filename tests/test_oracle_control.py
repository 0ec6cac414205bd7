"""Pins of the control-wrapper oracle (Sec. 4.1 action space, Sec. 4.2 100 Hz
physics under 20 Hz control).

Closed forms: repeated delta actions add up to k * a * delta and saturate at
the range's end; the gripper maps -1, 0, 1 to the range's ends and middle;
explicit Euler integration of a constant (v, w) base command sums a geometric
series in the complex plane; out-of-range and NaN actions act as clipped ones.
Physics: a PD drive that follows a ramp target reaches the ramp's speed, and
an arm joint settles at its stepped target.
"""
import numpy as np
import pytest

import oracle
from oracle import control as K
from paper_2412_13211_b300 import scenes as S
from helpers import cfg as mkcfg, env, scene_from_envs


def _spec(kind, act, scale, lo, hi, yaw=-1, A=None, steps=5):
    kind = np.asarray(kind, np.int32)
    return S.ControllerSpec(action_dim=A if A is not None else int(max(act) + 1), kind=kind,
                            action=np.asarray(act, np.int32), scale=np.asarray(scale, np.float32),
                            lo=np.asarray(lo, np.float32), hi=np.asarray(hi, np.float32), yaw_dof=yaw,
                            steps_per_action=steps)


def _run(spec, actions, t0, dt_c, precision="f64"):
    t = np.asarray(t0, np.float64)
    out = []
    for a in actions:
        t = K.controller(spec, a, t, dt_c, precision)
        out.append(t.copy())
    return np.array(out)


def test_delta_actions_add_up_and_saturate():
    spec = _spec([K.DELTA], [0], [0.1], [-1.0], [0.75])
    a = np.full((1, 1), 0.3)
    tr = _run(spec, [a] * 40, [[0.2]], 0.05)[:, 0, 0]
    k = np.arange(1, 41)
    step = 0.3 * float(np.float32(0.1))                  # the delta is stored in FP32
    free = 0.2 + k * step < 0.75
    np.testing.assert_allclose(tr[free], 0.2 + k[free] * step, rtol=0, atol=1e-12)
    assert (tr[~free] == np.float32(0.75)).all() and (~free).sum() > 5
    down = _run(spec, [-a] * 100, [[0.2]], 0.05)[:, 0, 0]
    assert down[-1] == -1.0 and np.all(np.diff(down) <= 0)


def test_actions_are_clipped_to_the_unit_box():
    spec = _spec([K.DELTA, K.DELTA, K.DELTA], [0, 1, 2], [0.1] * 3, [-9.0] * 3, [9.0] * 3)
    t0 = np.zeros((1, 3))
    got = K.controller(spec, np.array([[5.0, -7.0, np.nan]]), t0, 0.05, "f64")
    want = K.controller(spec, np.array([[1.0, -1.0, -1.0]]), t0, 0.05, "f64")
    assert np.array_equal(got, want)
    np.testing.assert_allclose(got, [[0.1, -0.1, -0.1]], rtol=0, atol=1e-7)   # delta stored in FP32


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_gripper_maps_the_unit_interval_onto_the_range(precision):
    spec = _spec([K.ABS, K.ABS], [0, 0], [0.0, 0.0], [0.0, 0.0], [0.05, 0.05])
    t0 = np.full((3, 2), 0.02)
    out = K.controller(spec, np.array([[-1.0], [0.0], [1.0]]), t0, 0.05, precision)
    hi = float(np.float32(0.05))
    assert out[0, 0] == 0.0 and out[2, 0] == np.asarray(hi, out.dtype)
    np.testing.assert_allclose(out[1], 0.5 * hi, rtol=1e-7)
    assert np.array_equal(out[:, 0], out[:, 1])          # one column drives both fingers


def test_base_velocity_integrates_along_the_previous_yaw():
    spec = _spec([K.BASE_X, K.BASE_Y, K.BASE_YAW, K.HOLD], [0, 0, 1, -1], [1.0, 1.0, 1.5, 0.0],
                 [-50.0, -50.0, -50.0, 0.0], [50.0, 50.0, 50.0, 1.0], yaw=2, A=2)
    dtc, av, aw, th0 = 0.05, 0.4, 0.6, 0.3
    v, w = av * 1.0, aw * np.float64(np.float32(1.5))
    n = 30
    tr = _run(spec, [np.array([[av, aw]])] * n, [[0.1, -0.2, th0, 0.7]], dtc)[:, 0]
    # k-th target: the sum of v dtc e^{i(th0 + j w dtc)} over j < k, a geometric series
    k = np.arange(1, n + 1)
    phi = w * dtc
    z = v * dtc * np.exp(1j * th0) * (1 - np.exp(1j * k * phi)) / (1 - np.exp(1j * phi))
    np.testing.assert_allclose(tr[:, 0], 0.1 + z.real, rtol=0, atol=1e-12)
    np.testing.assert_allclose(tr[:, 1], -0.2 + z.imag, rtol=0, atol=1e-12)
    np.testing.assert_allclose(tr[:, 2], th0 + k * phi, rtol=0, atol=1e-12)
    assert (tr[:, 3] == 0.7).all()                        # passive column untouched
    # turning in place leaves the position; driving straight keeps the heading
    spin = _run(spec, [np.array([[0.0, 1.0]])] * 4, [[0.1, -0.2, th0, 0.7]], dtc)[-1, 0]
    assert spin[0] == 0.1 and spin[1] == -0.2
    line = _run(spec, [np.array([[1.0, 0.0]])] * 4, [[0.0, 0.0, th0, 0.7]], dtc)[-1, 0]
    np.testing.assert_allclose(np.arctan2(line[1], line[0]), th0, atol=1e-12)
    np.testing.assert_allclose(np.hypot(line[0], line[1]), 4 * dtc, atol=1e-12)


def test_fp32_controller_tracks_fp64():
    sc, _ = S.make_config(6, num_envs=6)
    spec = sc.controller_spec()
    acts = sc.random_actions(20, spec.action_dim, amp=1.2)
    t32 = sc.targets0.astype(np.float32)
    t64 = sc.targets0.astype(np.float64)
    for a in acts:
        t32 = K.controller(spec, a, t32, K.control_dt(5, 0.01, "f32"), "f32")
        t64 = K.controller(spec, a, t64, K.control_dt(5, 0.01, "f64"), "f64")
        assert t32.dtype == np.float32
        np.testing.assert_allclose(t32, t64, rtol=0, atol=2e-6)
    held = spec.kind == K.HOLD
    assert held.sum() == 2 and np.array_equal(t32[:, held], sc.targets0[:, held])


def test_controller_spec_layouts():
    for idx, A, yaw in ((2, 8, -1), (3, 10, 2), (4, 8, -1), (6, 10, 4)):
        sc, _ = S.make_config(idx, num_envs=3)
        sp = sc.controller_spec()
        assert sp.action_dim == A and sp.yaw_dof == yaw and sp.steps_per_action == 5
        assert (sp.kind == K.DELTA).sum() == 7 and (sp.kind == K.ABS).sum() == 2
        assert sorted(set(sp.action[sp.kind != K.HOLD].tolist())) == list(range(A))
    with pytest.raises(ValueError):
        S.make_config(1, num_envs=2)[0].controller_spec()


def _robot_scene():
    e = env()
    S._add_robot(e, np.random.default_rng(3), (0.0, 0.0, 0.12), mobile_base=True)
    return scene_from_envs([e])


def test_base_follows_a_velocity_command():
    """A PD drive on a ramp target moves at the ramp's speed once the transient
    has decayed (kd/kp = 0.2 s of lag), along the commanded heading."""
    sc = _robot_scene()
    c = mkcfg(substeps=4, iterations=20)
    spec = sc.controller_spec()
    yaw0 = 0.5
    t = sc.targets0.astype(np.float32).copy()
    t[0, spec.yaw_dof] = yaw0
    st = sc.state()
    a = np.zeros((1, spec.action_dim), np.float32)
    a[0, spec.action[0]] = 0.3                           # v = 0.3 m/s, no turn
    hist = []
    for _ in range(50):                                   # 2.5 s
        st, t, status = K.control_step(sc, c, spec, st, a, t, "f64")
        hist.append(st[0][0, :2].copy())
    assert not status.any()
    vel = (hist[-1] - hist[-11]) / (10 * 0.05)
    np.testing.assert_allclose(np.hypot(*vel), 0.3, rtol=0.02)
    np.testing.assert_allclose(np.arctan2(vel[1], vel[0]), yaw0, atol=0.02)


def test_arm_joint_settles_at_the_stepped_target():
    """Two delta actions on the first arm joint (a revolute about world z on
    the base), then zero actions: the link's heading settles at 2 * 0.5 * 0.1
    rad."""
    sc = _robot_scene()
    c = mkcfg(substeps=4, iterations=20)
    spec = sc.controller_spec()
    t = sc.targets0.astype(np.float32).copy()
    st = sc.state()
    a = np.zeros((1, spec.action_dim), np.float32)
    j0 = int(np.nonzero(spec.kind == K.DELTA)[0][0])
    a[0, spec.action[j0]] = 0.5
    for k in range(30):
        st, t, _ = K.control_step(sc, c, spec, st, a if k < 2 else 0 * a, t, "f64")
    np.testing.assert_allclose(t[0, j0], 0.1, atol=1e-7)
    # the first link turns about world z (its hinge): its local y axis, horizontal, turns by the joint angle
    w, x, y, z = st[1][1]
    ly = np.array([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)])
    w, x, y, z = sc.quat[1].astype(np.float64)
    ly0 = np.array([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)])
    ang = np.arctan2(np.cross(ly0, ly)[2], ly0 @ ly)
    np.testing.assert_allclose(ang, 0.1, atol=2e-3)


def test_control_step_is_the_controller_then_the_physics_steps():
    sc, cfg = S.make_config(6, num_envs=2)
    spec = sc.controller_spec()
    a = sc.random_actions(1, spec.action_dim)[0]
    st, t, status = K.control_step(sc, cfg, spec, sc.state(), a, sc.targets0, "f32")
    t2 = K.controller(spec, a, sc.targets0, K.control_dt(5, cfg.dt), "f32")
    ref = sc.state()
    for _ in range(5):
        ref, _ = oracle.step(sc, cfg, ref, t2[None], 1, "f32")
    assert np.array_equal(t, t2)
    for x, y in zip(st, ref):
        assert np.array_equal(x, y)
