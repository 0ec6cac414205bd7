"""Pins of the oracle's reference gradients (forward-mode dual numbers).

Closed forms where the rollout is linear (free fall, a soft drive), and
central finite differences of the FP64 oracle (eps 1e-4) on the
differentiation workload (arm + boxes on a table, loss = squared distance of
one box to its goal). Directions where the rollout is not smooth between
+-eps (a contact or clamp switches) are detected by comparing two step
sizes and excluded, and their fraction is reported.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import cfg, env, scene_from_envs

G = 9.81


def test_free_fall_gradient_closed_form():
    """x_k = x0 + k h v0 + ..., so dL/dv0 . d = 2 (x_k - goal) . (k h d), and
    the mass does not enter."""
    e = env()
    e.body(S.SPHERE, (0.05,), 0.7, (0.1, -0.2, 50.0), linvel=(0.3, -0.1, 2.0))
    sc = scene_from_envs([e])
    c = cfg(substeps=3, iterations=4)
    n = 12
    goal = np.array([[0.5, 0.2, 49.0]])
    rng = np.random.default_rng(0)
    dvel = rng.normal(size=(2, 1, 6))
    dmass = np.array([[0.0], [1.0]])
    tg = np.zeros((n, 1, 1), np.float32)
    L, dL, st = oracle.loss_and_directional(sc, c, sc.state(), tg, n, [0], goal, dvel=dvel, dmass=dmass)
    out, _ = oracle.step(sc, c, sc.state(), tg, n, "f64")
    k, h = n * 3, 0.01 / 3
    r = out[0][0] - goal[0]
    assert abs(L[0] - r @ r) < 1e-12
    expect0 = 2 * r @ (k * h * dvel[0, 0, :3])
    expect1 = 2 * r @ (k * h * dvel[1, 0, :3])    # mass direction adds nothing
    np.testing.assert_allclose(dL[:, 0], [expect0, expect1], rtol=1e-11, atol=1e-11)


def _slider(m, k, d):
    e = env()
    e.body(S.BOX, (0.02, 0.02, 0.02), m, (0.0, 0.0, 1.0))
    e.joint(S.PRISMATIC, -1, 0, (0.0, 0.0, 1.0) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID, (k, d, 1e6), (-1.0, 1.0),
            [(0.0, 0.0, -1.0, 1.0)])
    return e


def test_soft_drive_gradient_matches_differentiated_recurrence():
    """A free slider on a soft drive follows the implicit-Euler recurrence
    exactly; its derivatives w.r.t. the targets and the mass are the
    derivatives of that recurrence (carried here as exact tangents)."""
    m, k, d = 0.25, 1000.0, 100.0
    sc = scene_from_envs([_slider(m, k, d)])
    Sub = 4
    c = cfg(substeps=Sub, iterations=3, gravity=(0.0, 0.0, 0.0))
    n = 10
    rng = np.random.default_rng(1)
    tg = rng.uniform(0.0, 0.04, size=(n, 1, 1)).astype(np.float32)
    goal = np.array([[0.01, 0.0, 1.0]])
    dtg = rng.normal(size=(2, n, 1, 1))
    dtg[1] = 0.0
    dmass = np.array([[0.0], [1.0]])
    L, dL, _ = oracle.loss_and_directional(sc, c, sc.state(), tg, n, [0], goal, dtargets=dtg, dmass=dmass)
    h = 0.01 / Sub
    mm = float(np.float32(m))
    # recurrence with tangents (x, v, dx, dv) for each direction
    res = []
    for kdir in range(2):
        x = v = dx = dv = 0.0
        dm = dmass[kdir, 0]
        for t in range(n):
            tau, dtau = float(tg[t, 0, 0]), dtg[kdir, t, 0, 0]
            for _ in range(Sub):
                den = 1 + h * d / mm + h * h * k / mm
                num = v - h * k / mm * (x - tau)
                # d(den)/dm and d(num)/dm
                dden = (-h * d / mm ** 2 - h * h * k / mm ** 2) * dm
                dnum = dv + h * k / mm ** 2 * (x - tau) * dm - h * k / mm * (dx - dtau)
                v_new = num / den
                dv = (dnum * den - num * dden) / den ** 2
                v = v_new
                x, dx = x + h * v, dx + h * dv
        res.append(2 * (x - goal[0, 0]) * dx)
    np.testing.assert_allclose(dL[:, 0], res, rtol=1e-9, atol=1e-12)


def _fd_case(sc, c, nsteps, seed):
    rng = np.random.default_rng(seed)
    E, B = sc.num_envs, sc.num_bodies
    md = max(sc.max_dof, 1)
    tg = sc.target_walk(nsteps, seed)
    dvel = rng.normal(size=(3, B, 6)) * 0.1
    dtg = np.zeros((3, nsteps, E, md))
    dtg[1] = rng.normal(size=(nsteps, E, md)) * 0.05
    dmass = np.zeros((3, B))
    dmass[2] = rng.normal(size=B) * sc.body_mass * 0.1
    dvel[1:] = 0.0
    return tg, dvel, dtg, dmass


def _fd(sc, c, tg, nsteps, dirs, eps):
    """Central differences of the FP64 rollout loss along each direction
    (velocities, targets and masses all perturbed in double)."""
    dvel, dtg, dmass = dirs
    out = []
    for k in range(dvel.shape[0]):
        vals = []
        for sgn in (1.0, -1.0):
            st = [a.astype(np.float64).copy() for a in sc.state()]
            st[2] += sgn * eps * dvel[k][:, :3]
            st[3] += sgn * eps * dvel[k][:, 3:]
            m = sc.body_mass.astype(np.float64) + sgn * eps * dmass[k]
            t2 = tg.astype(np.float64) + sgn * eps * dtg[k]
            L, _ = oracle.loss_value(sc, c, st, t2, nsteps, sc.goal_body, sc.goal_pos, mass=m)
            vals.append(L)
        out.append((vals[0] - vals[1]) / (2 * eps))
    return np.array(out)


@pytest.mark.parametrize("mode", [0, 1], ids=["coloured", "jacobi"])
@pytest.mark.parametrize("which", [0, 1, 2], ids=["velocity", "targets", "mass"])
def test_dual_gradient_matches_central_differences(which, mode, record_property):
    """Differentiation workload (arm pushing a box on a table), 8-step
    horizon, in both solver modes; directions in the initial velocities, the
    joint-target sequence or the masses. Central differences of the FP64
    oracle at eps = 1e-4 and eps/4: envs whose two differences disagree by
    more than 1% are not smooth within +-eps (a contact or clamp switches)
    and are excluded; the rest match the dual derivative to 2%. Counts are
    reported."""
    sc, c = S.make_config(4, num_envs=32)
    c.mode = mode
    nsteps = 8
    tg, dvel, dtg, dmass = _fd_case(sc, c, nsteps, 5)
    dirs = (dvel[which:which + 1], dtg[which:which + 1], dmass[which:which + 1])
    _, dL, status = oracle.loss_and_directional(sc, c, sc.state(), tg, nsteps, sc.goal_body, sc.goal_pos,
                                                dvel=dirs[0], dtargets=dirs[1], dmass=dirs[2])
    assert not status.any()
    eps = 1e-4
    fd1 = _fd(sc, c, tg, nsteps, dirs, eps)[0]
    fd2 = _fd(sc, c, tg, nsteps, dirs, eps / 4)[0]
    nonzero = np.abs(fd1) > 1e-8
    smooth = nonzero & (np.abs(fd1 - fd2) <= 1e-2 * np.abs(fd1))
    name = ["velocity", "targets", "mass"][which]
    record_property(f"nonzero_envs_{name}", int(nonzero.sum()))
    record_property(f"smooth_envs_{name}", int(smooth.sum()))
    assert nonzero.sum() >= 6 and smooth.sum() >= 0.5 * nonzero.sum()
    err = np.abs(dL[0] - fd1)
    assert (err[smooth] <= 2e-2 * np.abs(fd1[smooth])).all(), (dL[0], fd1)
    assert (np.abs(dL[0][~nonzero]) <= 1e-7).all()
