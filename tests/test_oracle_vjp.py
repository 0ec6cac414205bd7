"""Pins of the oracle's reverse-mode step adjoints (oracle.step_vjp).

The reverse-mode scalar records every arithmetic operation of one step with
its local partials and sweeps them backwards (Griewank and Walther's basic
operator-overloading scheme). These tests tie it to things other than
itself:
  * closed forms: free flight is linear in the state (x' = x + dt v + c,
    v' = v + dt g, omega' = omega), so its adjoints are known exactly;
  * the forward-mode dual numbers (themselves pinned against central
    differences and closed forms in test_oracle_grad.py): the chained FP64
    step adjoints contracted with a direction equal the dual directional
    derivative of the rollout loss, in both solver modes, since both follow
    the same FP64 branch decisions;
  * central differences of the FP64 step, element by element for every
    input of small scenes with resting contacts (normal and friction rows
    active), a swinging jointed chain with a drive and limits, and a Jacobi
    solve; an element whose difference changes between eps and eps/4 sits at
    a branch switch and is skipped (counted);
  * the FP32 primal: the FP32 form steps bit for bit like the FP32 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, cfg, env, scene_from_envs


def _rand_seed(sc, rng):
    B = sc.num_bodies
    return [rng.normal(size=(B, 3)), rng.normal(size=(B, 4)), rng.normal(size=(B, 3)), rng.normal(size=(B, 3))]


def test_free_flight_adjoint_closed_form():
    """No contact, no joint: x' = x + dt v + const, v' = v + dt g, omega' =
    omega. So dL/dx = w_x, dL/dv = dt w_x + w_v, dL/domega = w_omega (the
    quaternion seed set to zero), and the mass does not enter."""
    e = env()
    e.body(S.BOX, (0.05, 0.04, 0.03), 0.7, (0.1, -0.2, 50.0), quat=axis_angle((1, 2, 3), 0.4),
           linvel=(0.3, -0.1, 2.0), angvel=(0.5, -0.2, 0.1))
    e.body(S.SPHERE, (0.05,), 1.3, (5.0, 0.0, 40.0), linvel=(0.0, 1.0, 0.0))
    sc = scene_from_envs([e])
    c = cfg(substeps=3, iterations=4)
    rng = np.random.default_rng(3)
    w = _rand_seed(sc, rng)
    w[1][:] = 0.0
    r = oracle.step_vjp(sc, c, sc.state(), None, w, "f64")
    np.testing.assert_allclose(r.pos, w[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r.linvel, 0.01 * w[0] + w[2], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r.angvel, w[3], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r.mass, 0.0, atol=1e-13)
    np.testing.assert_allclose(r.quat, 0.0, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1], ids=["coloured", "jacobi"])
@pytest.mark.parametrize("idx,envs,nsteps", [(4, 16, 8), (2, 4, 3), (3, 4, 2)])
def test_chained_adjoints_equal_dual_directional_derivatives(idx, envs, nsteps, mode):
    """The FP64 step adjoints chained backwards along the rollout give the
    gradient of the goal loss; contracted with seeded directions in the
    initial velocities, the joint targets and the masses it equals the
    forward-mode dual derivative along each direction (same FP64 decisions,
    so to rounding)."""
    sc, c = S.make_config(idx, num_envs=envs)
    c.mode = mode
    rng = np.random.default_rng(11)
    B, E, md = sc.num_bodies, sc.num_envs, max(sc.max_dof, 1)
    tg = sc.target_walk(nsteps, 2)
    goal_body = np.where(sc.goal_body >= 0, sc.goal_body, 0)
    goal = sc.pos[sc.body_off[:-1] + goal_body].astype(np.float64) + rng.normal(size=(E, 3)) * 0.05
    dvel = rng.normal(size=(B, 6)) * 0.1
    dtg = rng.normal(size=(nsteps, E, md)) * 0.05
    dmass = rng.normal(size=B) * sc.body_mass * 0.1
    z = np.zeros
    _, dL, st = oracle.loss_and_directional(
        sc, c, sc.state(), tg, nsteps, goal_body, goal,
        dvel=np.stack([dvel, 0 * dvel, 0 * dvel]), dtargets=np.stack([0 * dtg, dtg, 0 * dtg]),
        dmass=np.stack([z(B), z(B), dmass]))
    g0, gtg, gm, xs, st2 = oracle.rollout_grad(
        sc, c, sc.state(), tg, nsteps, lambda x: oracle.goal_seed(sc, x[0], goal_body, goal), "f64")
    per_env = lambda a: np.add.reduceat(a, sc.body_off[:-1]) if B else a
    got = np.stack([
        per_env((g0[2] * dvel[:, :3]).sum(1) + (g0[3] * dvel[:, 3:]).sum(1)),
        (gtg * dtg[:, :, :sc.max_dof]).sum(axis=(0, 2)) if sc.max_dof else z(E),
        per_env(gm * dmass)])
    scale = np.abs(dL).max(axis=1, keepdims=True) + 1e-300
    assert (np.abs(got - dL) <= 1e-7 * scale + 1e-9 * np.abs(dL)).all(), (got, dL)
    assert np.abs(dL).max() > 0


def _tiny_scenes():
    """Small scenes whose every input is perturbed one by one."""
    out = []
    # a box resting on the plane (4 contact points, friction) with a sphere on top of it
    e = env()
    e.body(S.BOX, (0.1, 0.08, 0.05), 0.9, (0.0, 0.0, 0.0495), quat=axis_angle((0, 0, 1), 0.3),
           linvel=(0.2, 0.05, -0.1), angvel=(0.0, 0.0, 0.4))
    e.body(S.SPHERE, (0.04,), 0.3, (0.01, 0.0, 0.139), linvel=(0.0, 0.0, -0.3))
    out.append(("box_sphere_stack", e, cfg(substeps=2, iterations=6)))
    # a capsule sliding on a tilted static box
    e = env()
    e.static((0.0, 0.0, 0.1), (0.5, 0.5, 0.1), quat=axis_angle((1, 0, 0), 0.2))
    e.body(S.CAPSULE, (0.03, 0.08), 0.5, (0.0, 0.0, 0.235), quat=axis_angle((1, 0, 0), 0.2),
           linvel=(0.3, 0.0, 0.0))
    out.append(("capsule_on_incline", e, cfg(substeps=2, iterations=5)))
    # a two-link chain: revolute to the world with a drive, then a limited prismatic
    e = env()
    e.body(S.CAPSULE, (0.03, 0.15), 1.2, (0.15, 0.0, 1.0), angvel=(0.0, 0.5, 0.0))
    e.body(S.BOX, (0.03, 0.03, 0.03), 0.4, (0.35, 0.0, 1.0), linvel=(0.1, 0.0, 0.0))
    e.joint(S.REVOLUTE, -1, 0, (0.0, 0.0, 1.0) + axis_angle((0, 0, 1), np.pi / 2), (-0.15, 0.0, 0.0) +
            axis_angle((0, 0, 1), np.pi / 2), (200.0, 20.0, 100.0), (0.0, 0.0), [(0.1, 0.02, -3.0, 3.0)])
    e.joint(S.PRISMATIC, 0, 1, (0.15, 0.0, 0.0) + S.Q_ID, (-0.05, 0.0, 0.0) + S.Q_ID, (500.0, 50.0, 100.0),
            (0.0, 0.1), [(0.02, 0.0, 0.0, 0.1)])
    out.append(("driven_chain", e, cfg(substeps=3, iterations=8)))
    return out


def _fd_vjp(sc, c, state, tg, mass, w, eps):
    """sum_j w_j d out_j / d in_i by central differences for every input i."""
    def f(st, t, m):
        o, _ = oracle.step_f64x(sc, c, st, None if t is None else t[None], 1, mass=m)
        return sum(float((wi * oi).sum()) for wi, oi in zip(w, o))
    res = {}
    for name, k in (("pos", 0), ("quat", 1), ("linvel", 2), ("angvel", 3)):
        g = np.zeros(state[k].shape)
        for idx in np.ndindex(*state[k].shape):
            vals = []
            for sg in (1.0, -1.0):
                st = [a.copy() for a in state]
                st[k][idx] += sg * eps
                vals.append(f(st, tg, mass))
            g[idx] = (vals[0] - vals[1]) / (2 * eps)
        res[name] = g
    g = np.zeros(mass.shape)
    for i in range(mass.size):
        vals = []
        for sg in (1.0, -1.0):
            m = mass.copy()
            m[i] += sg * eps
            vals.append(f(state, tg, m))
        g[i] = (vals[0] - vals[1]) / (2 * eps)
    res["mass"] = g
    if tg is not None:
        g = np.zeros(tg.shape)
        for idx in np.ndindex(*tg.shape):
            vals = []
            for sg in (1.0, -1.0):
                t = tg.copy()
                t[idx] += sg * eps
                vals.append(f(state, t, mass))
            g[idx] = (vals[0] - vals[1]) / (2 * eps)
        res["targets"] = g
    return res


@pytest.mark.parametrize("mode", [0, 1], ids=["coloured", "jacobi"])
@pytest.mark.parametrize("case", range(3), ids=[n for n, _, _ in _tiny_scenes()])
def test_step_adjoint_elementwise_matches_central_differences(case, mode, record_property):
    name, e, c = _tiny_scenes()[case]
    c.mode = mode
    sc = scene_from_envs([e])
    rng = np.random.default_rng(case)
    state = [a.astype(np.float64) for a in sc.state()]
    tg = sc.targets0.astype(np.float64).reshape(1, -1) if sc.max_dof else None
    mass = sc.body_mass.astype(np.float64)
    w = _rand_seed(sc, rng)
    r = oracle.step_vjp(sc, c, state, tg, w, "f64")
    assert not r.status.any()
    fd1 = _fd_vjp(sc, c, state, tg, mass, w, 1e-6)
    fd2 = _fd_vjp(sc, c, state, tg, mass, w, 2.5e-7)
    got = dict(pos=r.pos, quat=r.quat, linvel=r.linvel, angvel=r.angvel, mass=r.mass)
    if tg is not None:
        got["targets"] = r.targets
    skipped = total = 0
    for k, g in got.items():
        a, b = fd1[k], fd2[k]
        scale = max(np.abs(a).max(), 1e-6)
        smooth = np.abs(a - b) <= 1e-6 * scale + 1e-4 * np.abs(a)
        skipped += int((~smooth).sum())
        total += a.size
        err = np.abs(g - a)
        assert (err[smooth] <= 1e-5 * scale + 1e-4 * np.abs(a[smooth])).all(), (k, g, a)
    record_property("skipped_elements", skipped)
    assert skipped <= total // 10


def test_fp32_form_steps_like_the_fp32_oracle():
    sc, c = S.make_config(3, num_envs=6)
    tg = sc.target_walk(1)
    o, _ = oracle.step(sc, c, sc.state(), tg, 1, "f32")
    r = oracle.step_vjp(sc, c, sc.state(), tg[0], _rand_seed(sc, np.random.default_rng(0)), "f32")
    for a, b in zip(o, r.out):
        assert np.array_equal(a.view(np.int32), b.view(np.int32))


def test_fp32_and_fp64_adjoints_agree_on_a_contact_free_arm():
    """The arm of the manipulator scene swinging in free space (no contact):
    a smooth step, so the FP32-primal and FP64 adjoints agree closely."""
    sc, c = S.make_config(2, num_envs=2)
    keep = [np.arange(sc.body_off[e], sc.body_off[e + 1]) for e in range(sc.num_envs)]
    st = [a.copy() for a in sc.state()]
    st[0][:, 2] += 5.0          # lift everything: nothing touches the counter or the plane
    for e in range(sc.num_envs):   # spread the objects apart in the air
        st[0][keep[e][9:], 0] += 2.0 * np.arange(1, len(keep[e]) - 8)
    tg = sc.target_walk(1)[0]
    w = _rand_seed(sc, np.random.default_rng(4))
    r32 = oracle.step_vjp(sc, c, st, tg, w, "f32")
    r64 = oracle.step_vjp(sc, c, st, tg, w, "f64")
    det = oracle.detect(sc, c, st[0], st[1])
    assert det.contact_count.sum() == 0
    for k in ("pos", "quat", "linvel", "angvel", "targets", "mass"):
        a, b = getattr(r32, k), getattr(r64, k)
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max() + 1e-9, k
