"""Pins of the oracle's contact report (pairwise contact forces, the robot's
cumulative collision force and the grasp indicator that the paper's subtask
conditions and event labels use, Sec. 3.3 and Appendix A.4-A.5).

At rest a body's velocity is zero after every solve, so its net contact
impulse per substep cancels gravity exactly: its net contact force is its
weight, whatever the solver's convergence. An isolated impact gives equal and
opposite forces. A box held between two drive-pushed fingers against gravity
hangs on friction: the fingers carry its weight between them.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, cfg, env, scene_from_envs

G = 9.81
QZ180 = axis_angle((0.0, 0.0, 1.0), np.pi)


def _report(sc, c, nsteps, flags, fingers=(-1, -1), target=-1, targets=None, precision="f64", **kw):
    E = sc.num_envs
    return oracle.step_report(sc, c, sc.state(), targets, nsteps, np.asarray(flags, np.int32),
                              np.tile(np.asarray(fingers, np.int32), (E, 1)), np.full(E, target, np.int32),
                              precision=precision, **kw)


def test_resting_stack_each_body_carries_its_weight():
    """Box on box on the plane: each body's net contact force is m g upwards."""
    e = env()
    e.body(S.BOX, (0.125, 0.125, 0.0625), 2.0, (0.0, 0.0, 0.0625))
    e.body(S.BOX, (0.0625, 0.0625, 0.0625), 0.5, (0.0, 0.0, 0.1875))
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=30)
    out, st, rep = _report(sc, c, 200, [0, 0])
    assert not st.any()
    np.testing.assert_allclose(rep.body_force, [[0, 0, 2.0 * G], [0, 0, 0.5 * G]], rtol=1e-6, atol=1e-6)


def test_impact_forces_equal_and_opposite():
    e = env()
    e.body(S.SPHERE, (0.05,), 0.3, (0.0, 0.0, 1.0), linvel=(1.0, 0.0, 0.0))
    e.body(S.SPHERE, (0.07,), 0.9, (0.125, 0.01, 1.0), linvel=(-0.5, 0.0, 0.0))
    sc = scene_from_envs([e])
    c = cfg(substeps=2, iterations=10, gravity=(0.0, 0.0, 0.0))
    peak = 0.0
    for n in (1, 2, 3):
        out, _, rep = _report(sc, c, n, [0, 0])
        assert np.array_equal(rep.body_force[0], -rep.body_force[1])
        peak = max(peak, np.abs(rep.body_force).max())
    assert peak > 1.0   # they did collide
    # the impulse over the step matches the momentum change of either sphere
    v0 = sc.linvel.astype(np.float64)
    out1, _, rep1 = _report(sc, c, 1, [0, 0])
    m = sc.body_mass.astype(np.float64)              # the stored (f32) masses
    np.testing.assert_allclose(rep1.body_force[1] * 0.01, m[1] * (out1[2][1] - v0[1]), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(rep1.body_force[0] * 0.01, m[0] * (out1[2][0] - v0[0]), rtol=1e-9, atol=1e-12)


def _robot_on(support):
    """A 'robot link' box resting on a static box, a plain dynamic box, or the plane."""
    e = env()
    if support == "static":
        e.static((0.0, 0.0, 0.25), (0.3, 0.3, 0.25))
        z0 = 0.5
    elif support == "dynamic":
        e.body(S.BOX, (0.2, 0.2, 0.05), 3.0, (0.0, 0.0, 0.05))
        z0 = 0.1
    else:
        z0 = 0.0
    e.body(S.BOX, (0.1, 0.1, 0.05), 1.5, (0.0, 0.0, z0 + 0.05))
    return e


@pytest.mark.parametrize("support,counts", [("static", True), ("dynamic", True), ("plane", False)])
def test_cumulative_robot_force_adds_the_support_force_per_step(support, counts):
    e = _robot_on(support)
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=30)
    flags = [0] * (sc.num_bodies - 1) + [1]
    # settle, then accumulate k more steps from the settled state
    out, _, rep0 = _report(sc, c, 150, flags)
    k = 20
    st = [np.asarray(a, np.float64) for a in out]
    _, _, rep = oracle.step_report(sc, c, st, None, k, np.asarray(flags, np.int32), np.full((1, 2), -1, np.int32),
                                   np.full(1, -1, np.int32), precision="f64")
    expect = k * 1.5 * G if counts else 0.0
    assert abs(rep.robot_force[0] - expect) <= 1e-5 * max(expect, 1.0)
    assert rep0.robot_force[0] >= 0.0


def test_robot_contacts_with_itself_and_the_target_do_not_count():
    """Robot link on a robot link, and a robot end-effector link on the target:
    no collision force; the target force is the ee link's weight pressing down."""
    for flags_lower, target in ((1, -1), (0, 0)):
        e = _robot_on("dynamic")
        sc = scene_from_envs([e])
        c = cfg(substeps=4, iterations=30)
        flags = [flags_lower, 1 | 2]
        out, _, _ = _report(sc, c, 150, flags, target=target)
        st = [np.asarray(a, np.float64) for a in out]
        _, _, rep = oracle.step_report(sc, c, st, None, 10, np.asarray(flags, np.int32),
                                       np.full((1, 2), -1, np.int32), np.full(1, target, np.int32),
                                       precision="f64")
        # the lower box rests on the plane (not counted) and the upper counts nothing
        assert abs(rep.robot_force[0]) < 1e-9
        if target == 0:
            np.testing.assert_allclose(rep.target_force[0], [0.0, 0.0, -1.5 * G], rtol=1e-6, atol=1e-6)
        else:
            assert np.array_equal(rep.target_force[0], [0.0, 0.0, 0.0])


def _gripper(gravity=True, k=1000.0):
    """Two box fingers on prismatic joints along x (the right one mirrored),
    driven into a 6 cm box between them."""
    e = env()
    e.body(S.BOX, (0.03, 0.03, 0.03), 0.2, (0.0, 0.0, 1.0))                  # 0: target
    e.body(S.BOX, (0.01, 0.02, 0.02), 0.1, (-0.05, 0.0, 1.0))                 # 1: left finger
    e.body(S.BOX, (0.01, 0.02, 0.02), 0.1, (0.05, 0.0, 1.0), QZ180)           # 2: right finger
    gains = (k, 100.0, 200.0)
    e.joint(S.PRISMATIC, -1, 1, (-0.1, 0.0, 1.0) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID, gains, (-1.0, 1.0),
            [(0.05, 0.0, -1.0, 1.0)])
    e.joint(S.PRISMATIC, -1, 2, (0.1, 0.0, 1.0) + tuple(QZ180), (0.0, 0.0, 0.0) + S.Q_ID, gains, (-1.0, 1.0),
            [(0.05, 0.0, -1.0, 1.0)])
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=30, gravity=(0.0, 0.0, -G if gravity else 0.0))
    return sc, c


def _squeeze(n):
    return np.full((n, 1, 2), 0.1, np.float32)     # both fingers driven to the box centre


def test_grasp_holds_box_weight_by_friction():
    sc, c = _gripper()
    n = 150
    out, st, rep = _report(sc, c, n, [0, 3, 3], fingers=(1, 2), target=0, targets=_squeeze(n))
    assert not st.any()
    assert rep.grasped[0] == 1
    FL, FR = rep.finger_force[0]
    # the box hangs: the fingers carry its weight (up to the slow creep of an
    # iterative friction solve), and squeeze it symmetrically
    m = float(sc.body_mass[0])
    assert abs((FL[2] + FR[2]) + m * G) < 0.01 * m * G
    assert FL[0] < -10.0 and FR[0] > 10.0 and abs(FL[0] + FR[0]) < 1e-3
    # held, not falling (a free fall would have dropped 11 m)
    assert abs(out[0][0][2] - 1.0) < 1e-2 and np.abs(out[2][0]).max() < 1e-2
    # target force: the fingers (end-effector links) hold the box up
    np.testing.assert_allclose(rep.target_force[0], -(FL + FR), rtol=1e-9, atol=1e-9)


def test_grasp_decision_thresholds():
    """grasped flips where f_min crosses the finger force and where the angle
    limit crosses the angle between a finger's force and its opening direction."""
    sc, c = _gripper()
    n = 150
    out, _, rep = _report(sc, c, n, [0, 3, 3], fingers=(1, 2), target=0, targets=_squeeze(n))
    xs = (out[0][1], out[0][2])

    def angle(f):
        F, o = rep.finger_force[0][f], xs[f] - xs[1 - f]
        return np.degrees(np.arccos(F @ o / (np.linalg.norm(F) * np.linalg.norm(o))))
    ang = max(angle(0), angle(1))          # both fingers must pass
    assert 0.0 < ang < 30.0
    fmag = min(np.linalg.norm(f) for f in rep.finger_force[0])
    for kw, expect in ((dict(grasp_min_force=fmag * 0.99), 1), (dict(grasp_min_force=fmag * 1.01), 0),
                       (dict(grasp_max_angle_deg=ang + 0.05), 1), (dict(grasp_max_angle_deg=ang - 0.05), 0)):
        _, _, r = _report(sc, c, n, [0, 3, 3], fingers=(1, 2), target=0, targets=_squeeze(n), **kw)
        assert r.grasped[0] == expect, kw


def test_no_grasp_with_one_finger_or_open_fingers():
    sc, c = _gripper(gravity=False)
    n = 100
    one = np.full((n, 1, 2), 0.1, np.float32)
    one[:, 0, 1] = -0.2                               # right finger pulled away
    _, _, rep = _report(sc, c, n, [0, 3, 3], fingers=(1, 2), target=0, targets=one)
    assert rep.grasped[0] == 0
    assert np.linalg.norm(rep.finger_force[0][1]) == 0.0
    opened = np.full((n, 1, 2), -0.2, np.float32)
    _, _, rep = _report(sc, c, n, [0, 3, 3], fingers=(1, 2), target=0, targets=opened)
    assert rep.grasped[0] == 0 and np.abs(rep.finger_force[0]).max() == 0.0


def test_report_does_not_change_the_step():
    sc, cf = S.make_config(3, num_envs=3)
    tg = sc.target_walk(3)
    flags = np.zeros(sc.num_bodies, np.int32)
    a, sa = oracle.step(sc, cf, sc.state(), tg, 3, "f32")
    b, sb, rep = oracle.step_report(sc, cf, sc.state(), tg, 3, flags, np.full((3, 2), -1, np.int32),
                                    np.full(3, -1, np.int32), precision="f32")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(sa, sb)
