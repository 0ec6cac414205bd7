"""The CUDA contact report (msh_set_report) against the oracle's.

Forces derive from the solver's lambdas, so they agree to the solver's FP32
tolerance: the step's velocity tolerance (1e-4 m/s) times a body's mass over
dt bounds a force difference by about 0.01 N per kg; the tests allow 0.05 N
plus 1e-3 relative. Grasp decisions are compared where both sides' margins
to the force and angle thresholds exceed that tolerance; elsewhere both
answers are valid. One step is compared from a common start state so that
trajectory divergence does not enter.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu

ATOL, RTOL = 0.05, 1e-3


def _gpu(sc, cfg, state, targets, nsteps, spec, **kw):
    import torch
    from paper_2412_13211_b300.sim import MshSim
    sim = MshSim(sc, cfg, **kw)
    sim.set_state(*state)
    sim.set_report(*spec)
    tg = torch.as_tensor(np.asarray(targets, np.float32)).cuda() if targets is not None else None
    for t in range(nsteps):
        sim.step(tg[t] if tg is not None else None)
    out = sim.state_numpy(), sim.report(), sim.status()
    sim.close()
    return out


def _oracle(sc, cfg, state, targets, nsteps, spec):
    flags, fingers, target = spec
    return oracle.step_report(sc, cfg, state, targets, nsteps, flags, fingers, target, precision="f32")


def _close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) <= ATOL + RTOL * np.abs(b)


def _settled_state(sc, cfg, targets, n):
    out, _ = oracle.step(sc, cfg, sc.state(), targets, n, "f32")
    return [np.ascontiguousarray(a, np.float32) for a in out]


@pytest.mark.parametrize("idx,envs", [(2, 16), (4, 16), (3, 8), (6, 8)])
def test_report_matches_oracle_one_step(idx, envs):
    sc, cfg = S.make_config(idx, num_envs=envs)
    spec = sc.report_spec()
    tg = sc.target_walk(21)
    st = _settled_state(sc, cfg, tg, 20)
    (gs, grep, gstat), (os_, ostat, orep) = _gpu(sc, cfg, st, tg[20:], 1, spec), _oracle(sc, cfg, st, tg[20:], 1, spec)
    assert not gstat.any() and not ostat.any()
    assert _close(grep["body_force"], orep.body_force).all()
    assert _close(grep["target_force"], orep.target_force).all()
    assert _close(grep["finger_force"], orep.finger_force).all()
    assert _close(grep["robot_force"], orep.robot_force).all()
    assert np.abs(orep.body_force).max() > 1.0           # there are contacts to compare


def _gripper_batch(ks):
    """Envs of two drive-pushed fingers squeezing a box, with drive stiffness ks."""
    from helpers import axis_angle, env, scene_from_envs
    qz = axis_angle((0.0, 0.0, 1.0), np.pi)
    envs = []
    for k in ks:
        e = env()
        e.body(S.BOX, (0.03, 0.03, 0.03), 0.2, (0.0, 0.0, 1.0))
        e.body(S.BOX, (0.01, 0.02, 0.02), 0.1, (-0.05, 0.0, 1.0))
        e.body(S.BOX, (0.01, 0.02, 0.02), 0.1, (0.05, 0.0, 1.0), qz)
        g = (k, 100.0, 200.0)
        e.joint(S.PRISMATIC, -1, 1, (-0.1, 0.0, 1.0) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID, g, (-1.0, 1.0),
                [(0.05, 0.0, -1.0, 1.0)])
        e.joint(S.PRISMATIC, -1, 2, (0.1, 0.0, 1.0) + tuple(qz), (0.0, 0.0, 0.0) + S.Q_ID, g, (-1.0, 1.0),
                [(0.05, 0.0, -1.0, 1.0)])
        e.goal_body = 0
        envs.append(e)
    return scene_from_envs(envs)


def test_grasp_indicator_matches_oracle():
    from helpers import cfg
    ks = [5.0, 20.0, 100.0, 400.0, 1000.0, 3000.0]
    sc = _gripper_batch(ks)
    c = cfg(substeps=4, iterations=30)
    spec = sc.report_spec()
    assert (spec[1] == [1, 2]).all() and (spec[2] == 0).all()
    tg = np.full((61, sc.num_envs, 2), 0.1, np.float32)
    st = _settled_state(sc, c, tg, 60)
    (gs, grep, _), (_, _, orep) = _gpu(sc, c, st, tg[60:], 1, spec), _oracle(sc, c, st, tg[60:], 1, spec)
    assert _close(grep["finger_force"], orep.finger_force).all()
    # decisions with a clear margin must agree; the stiff drives do grasp
    fmag = np.linalg.norm(orep.finger_force, axis=2).min(axis=1)
    clear = np.abs(fmag - 0.5) > ATOL + RTOL * fmag
    assert clear.sum() >= 4
    assert np.array_equal(grep["grasped"][clear], orep.grasped[clear])
    assert orep.grasped[-1] == 1


def test_report_identical_across_forms():
    sc, cfg = S.make_config(2, num_envs=8)
    spec = sc.report_spec()
    tg = sc.target_walk(3)
    st = sc.state()
    res = []
    for kw in (dict(exec_form="fused"), dict(exec_form="plain"), dict(exec_form="substep"),
               dict(exec_form="fused", threads_per_env=16, use_graph=True)):
        _, rep, _ = _gpu(sc, cfg, st, tg, 3, spec, **kw)
        res.append(rep)
    for r in res[1:]:
        for k in r:
            assert np.array_equal(r[k], res[0][k]), k


def test_robot_force_accumulates_and_report_can_be_turned_off():
    import torch
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(3, num_envs=8)
    tg = torch.as_tensor(sc.target_walk(6)).cuda()
    sim = MshSim(sc, cfg)
    out = sim.set_report(*sc.report_spec())
    acc = np.zeros(sc.num_envs)
    for t in range(3):
        before = out["robot_force"].cpu().numpy().copy()
        sim.step(tg[t])
        after = out["robot_force"].cpu().numpy()
        assert (after >= before).all()
        acc = after
    sim.reset_robot_force()
    assert not out["robot_force"].any()
    sim.clear_report()
    sim.step(tg[3])
    assert not out["robot_force"].any()        # no longer written
    assert acc.max() >= 0.0
    sim.close()


def test_recorded_steps_do_not_write_the_report():
    import torch
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(4, num_envs=4)
    sim = MshSim(sc, cfg)
    out = sim.set_report(*sc.report_spec())
    out["robot_force"].fill_(-1.0)
    sim.set_tape(2)
    tg = torch.as_tensor(sc.target_walk(2)).cuda()
    sim.step(tg[0])
    assert (out["robot_force"].cpu().numpy() == -1.0).all()
    sim.set_tape(-1)
    sim.close()
