"""Rigid-motion equivariance of the oracle's narrowphase (FP64 on FP32-stored
poses). Moving both shapes of a pair by one rigid motion (a rotation about a
pivot near them, then a translation) must leave the manifold unchanged in
each body's own frame and turn its normal with the rotation: the same
contacts in the same order, the same separations and body-local anchors, and
the rotated normal. This holds for every one of the six pairs of dynamic
shape types, whatever the features each routine picks, so a routine that
uses an absolute position or orientation where a relative one belongs, a
transposed rotation when it takes an anchor into the body frame, or a normal
left in a body frame fails it.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, cfg, env, quat_mul, scene_from_envs

TYPES = {S.SPHERE: "sphere", S.CAPSULE: "capsule", S.BOX: "box"}


def _rot(q):
    w, x, y, z = (float(v) for v in q)
    U = np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])
    return np.eye(3) + 2.0 * w * U + 2.0 * U @ U


def _dims(rng, t):
    if t == S.SPHERE:
        return (rng.uniform(0.03, 0.08),), 0.08
    if t == S.CAPSULE:
        r, L = rng.uniform(0.02, 0.05), rng.uniform(0.04, 0.12)
        return (r, L), r + L
    h = rng.uniform(0.03, 0.09, 3)
    return tuple(h), float(np.linalg.norm(h))


def _pair(rng, ta, tb, pos_a, q_a, q_b, u, frac):
    da, ra = _dims(rng, ta)
    db, rb = _dims(rng, tb)
    pos_b = np.asarray(pos_a) + u * frac * (ra + rb)
    e = env()
    e.body(ta, da, 1.0, tuple(pos_a), tuple(q_a))
    e.body(tb, db, 1.0, tuple(pos_b), tuple(q_b))
    return e, (ta, da), (tb, db)


def _detect(sc):
    return oracle.detect(sc, cfg(max_pairs=16, max_contacts=32), sc.pos, sc.quat, precision="f64")


def _moved(e, qm, pivot, shift):
    """The same two bodies after x -> R(qm)(x - pivot) + pivot + shift, q -> qm q."""
    R = _rot(qm)
    m = env()
    for (shape, dims, mass, pos, quat, _, _) in e.bodies:
        x = R @ (np.asarray(pos, float) - pivot) + pivot + shift
        q = quat_mul(qm, quat)
        q = q / np.linalg.norm(q)
        m.body(shape, dims[:3], mass, tuple(x), tuple(q))
    return m


@pytest.mark.parametrize("ta,tb", list(itertools.combinations_with_replacement(sorted(TYPES), 2)),
                         ids=lambda t: TYPES[t] if isinstance(t, int) else str(t))
def test_manifold_is_equivariant_under_rigid_motion(ta, tb):
    rng = np.random.default_rng(1000 + 10 * ta + tb)
    checked = points = 0
    for _ in range(150):
        q_a = axis_angle(rng.normal(size=3), rng.uniform(0.0, np.pi))
        q_b = axis_angle(rng.normal(size=3), rng.uniform(0.0, np.pi))
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos_a = np.array([rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0), 3.0])
        e, _, _ = _pair(rng, ta, tb, pos_a, q_a, q_b, u, rng.uniform(0.45, 0.95))
        sc = scene_from_envs([e])
        d = _detect(sc)
        n = int(d.contact_count[0])
        if n == 0:
            continue
        qm = axis_angle(rng.normal(size=3), rng.uniform(0.3, np.pi))
        shift = np.array([rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(0.0, 1.0)])
        pivot = sc.pos[:2].astype(np.float64).mean(axis=0)
        sc2 = scene_from_envs([_moved(e, qm, pivot, shift)])
        d2 = _detect(sc2)
        assert int(d2.contact_count[0]) == n
        assert np.array_equal(d2.contact_ids[0, :n], d.contact_ids[0, :n])
        R = _rot(qm)
        g, g2 = d.contact_geom[0, :n], d2.contact_geom[0, :n]
        # the stored FP32 poses of the moved pair are the exact motion to ~1e-7 m
        np.testing.assert_allclose(g2[:, :3], g[:, :3] @ R.T, atol=2e-5)
        np.testing.assert_allclose(g2[:, 3:9], g[:, 3:9], atol=2e-6)
        np.testing.assert_allclose(g2[:, 9], g[:, 9], atol=2e-6)
        checked += 1
        points += n
    # enough configurations in contact for the pin to mean something
    assert checked >= 30, checked
    if ta == S.BOX and tb == S.BOX:
        assert points > checked   # multi-point manifolds among them


def test_a_transposed_anchor_frame_breaks_the_pin():
    """The pin is not vacuous: the anchors taken into the body frame with the
    rotation instead of its transpose (a plausible mistake) are not invariant
    under the same motions."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(20):
        q_a = axis_angle(rng.normal(size=3), rng.uniform(0.5, np.pi))
        e, _, _ = _pair(rng, S.BOX, S.SPHERE, np.array([0.0, 0.0, 3.0]), q_a, (1.0, 0.0, 0.0, 0.0),
                        np.array([0.0, 0.0, 1.0]), 0.6)
        sc = scene_from_envs([e])
        d = _detect(sc)
        if d.contact_count[0] == 0:
            continue
        qm = axis_angle(rng.normal(size=3), rng.uniform(0.5, np.pi))
        sc2 = scene_from_envs([_moved(e, qm, sc.pos[0].astype(np.float64), np.zeros(3))])
        d2 = _detect(sc2)
        Ra, Ra2 = _rot(sc.quat[0]), _rot(sc2.quat[0])
        wa = sc.pos[0] + Ra @ d.contact_geom[0, 0, 3:6]           # world anchor before the motion
        wa2 = sc2.pos[0] + Ra2 @ d2.contact_geom[0, 0, 3:6]
        wrong, wrong2 = Ra @ (wa - sc.pos[0]), Ra2 @ (wa2 - sc2.pos[0])   # R instead of R^T
        worst = max(worst, float(np.abs(wrong2 - wrong).max()))
    assert worst > 1e-3
