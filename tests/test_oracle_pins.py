"""Pins of the CPU oracle to closed forms, invariants and brute force.

Each test checks the oracle against something other than itself: the exact
discrete solution of the integrator, a hand-derived projected Gauss-Seidel
iteration, conservation laws, an independent geometric construction, or a
brute-force enumeration. These run without a GPU.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, cfg, env, quat_mul, quat_rotate, scene_from_envs

G = 9.81


# --------------------------------------------------------------------------
# integrator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("substeps", [1, 3])
def test_free_fall_matches_discrete_closed_form(substeps):
    """Symplectic Euler without contacts: v_k = v0 + k h g and
    x_k = x0 + k h v0 + h^2 g k(k+1)/2 after k substeps."""
    e = env()
    x0, v0 = np.array([0.1, -0.2, 50.0]), np.array([0.3, -0.1, 2.0])
    e.body(S.SPHERE, (0.05,), 0.7, tuple(x0), linvel=tuple(v0))
    e.body(S.BOX, (0.1, 0.05, 0.02), 1.3, (5.0, 5.0, 40.0), linvel=(-1.0, 0.5, 0.0))
    sc = scene_from_envs([e])
    c = cfg(substeps=substeps, iterations=5)
    n = 40
    out, status = oracle.step(sc, c, sc.state(), None, nsteps=n, precision="f64")
    assert status[0] == 0
    h, k = 0.01 / substeps, n * substeps
    g = np.array([0.0, 0.0, -G])
    for i in range(2):
        xi, vi = sc.pos[i].astype(np.float64), sc.linvel[i].astype(np.float64)
        v = vi + k * h * g
        x = xi + k * h * vi + h * h * g * k * (k + 1) / 2
        np.testing.assert_allclose(out[2][i], v, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(out[0][i], x, rtol=1e-12, atol=1e-12)
    # FP32 mode agrees with the closed form to single-precision rounding
    out32, _ = oracle.step(sc, c, sc.state(), None, nsteps=n, precision="f32")
    x0, v0 = sc.pos[0].astype(np.float64), sc.linvel[0].astype(np.float64)
    np.testing.assert_allclose(out32[0][0], x0 + k * h * v0 + h * h * g * k * (k + 1) / 2, atol=2e-5)


def test_torque_free_rotation_angle_is_discrete_closed_form():
    """Spin about a principal axis with no contacts: w is unchanged and each
    substep turns the body by exactly 2 atan(h|w|/2) (normalised
    q + h/2 (0,w) q); |q| stays 1."""
    e = env()
    w = 3.0
    e.body(S.BOX, (0.1, 0.2, 0.3), 1.0, (0.0, 0.0, 10.0), angvel=(0.0, 0.0, w))
    sc = scene_from_envs([e])
    c = cfg(substeps=2, iterations=3, gravity=(0.0, 0.0, 0.0))
    n = 100
    out, _ = oracle.step(sc, c, sc.state(), None, nsteps=n, precision="f64")
    h = 0.01 / 2
    phi = 2 * n * 2 * np.arctan(h * w / 2)
    q = out[1][0]
    assert np.array_equal(out[3][0], [0.0, 0.0, w])
    ang = 2 * np.arctan2(q[3], q[0])
    assert abs(np.angle(np.exp(1j * (ang - phi)))) < 1e-10
    out32, _ = oracle.step(sc, c, sc.state(), None, nsteps=1000, precision="f32")
    assert abs(np.linalg.norm(out32[1][0].astype(np.float64)) - 1) < 1e-6


# --------------------------------------------------------------------------
# contact normal rows
# --------------------------------------------------------------------------
@pytest.mark.parametrize("substeps", [1, 4])
def test_resting_sphere_normal_impulse_is_mg(substeps):
    """A sphere touching the plane: one projected GS row cancels gravity exactly
    (lambda/h = m g), so the sphere stays at rest with zero velocity."""
    e = env()
    e.body(S.SPHERE, (0.0625,), 0.75, (0.25, -0.125, 0.0625))   # exact in f32
    sc = scene_from_envs([e])
    out, _ = oracle.step(sc, cfg(substeps=substeps, iterations=1), sc.state(), None, nsteps=50,
                         precision="f64")
    assert abs(out[0][0][2] - 0.0625) < 1e-12
    assert np.abs(out[2][0]).max() < 1e-12


def test_box_on_plane_four_corner_contacts_and_rest():
    e = env()
    hx, hy, hz = 0.125, 0.25, 0.0625
    q = (1.0, 0.0, 0.0, 0.0)
    e.body(S.BOX, (hx, hy, hz), 2.0, (0.25, 0.125, hz - 2.0 ** -10), q)
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=20)
    d = oracle.detect(sc, c, sc.pos, sc.quat, precision="f64")
    assert d.contact_count[0] == 4
    g = d.contact_geom[0, :4]
    np.testing.assert_allclose(g[:, :3], np.tile([0, 0, -1.0], (4, 1)))
    np.testing.assert_allclose(g[:, 9], -2.0 ** -10, atol=1e-15)
    corners = {tuple(np.round(np.array([sx * hx, sy * hy, -hz]), 12)) for sx in (-1, 1) for sy in (-1, 1)}
    got = {tuple(np.round(r, 12)) for r in g[:, 3:6]}
    assert got == corners
    out, _ = oracle.step(sc, c, sc.state(), None, nsteps=100, precision="f64")
    assert np.abs(out[2][0]).max() < 1e-3
    assert abs(out[0][0][2] - hz) < 2e-3


# --------------------------------------------------------------------------
# friction
# --------------------------------------------------------------------------
@pytest.mark.parametrize("theta_deg", [20.0, 40.0])
def test_box_on_incline_sticks_iff_tan_below_mu(theta_deg):
    """Gravity tilted by theta on a flat plane (mu = 0.5): rest iff
    tan(theta) <= mu, else acceleration g (sin(theta) - mu cos(theta))."""
    th = np.deg2rad(theta_deg)
    e = env()
    e.body(S.BOX, (0.1, 0.1, 0.03), 1.0, (0.0, 0.0, 0.03))
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=30, friction=0.5,
            gravity=(G * np.sin(th), 0.0, -G * np.cos(th)))
    st = sc.state()
    s50, _ = oracle.step(sc, c, st, None, nsteps=50, precision="f64")
    s100, _ = oracle.step(sc, c, s50, None, nsteps=50, precision="f64")
    if np.tan(th) <= 0.5:
        assert np.abs(s100[2][0]).max() < 1e-3
    else:
        a = (s100[2][0][0] - s50[2][0][0]) / 0.5
        expect = G * (np.sin(th) - 0.5 * np.cos(th))
        assert abs(a - expect) < 0.02 * expect


# --------------------------------------------------------------------------
# momentum
# --------------------------------------------------------------------------
def _momenta(sc, st):
    m = sc.body_mass.astype(np.float64)
    P = (m[:, None] * st[2]).sum(0)
    L = (m[:, None] * np.cross(st[0], st[2])).sum(0)
    return P, L


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_two_sphere_impact_conserves_momentum(mu):
    e = env()
    e.body(S.SPHERE, (0.05,), 0.4, (0.0, 0.0, 1.0), linvel=(2.0, 0.3, 0.0))
    e.body(S.SPHERE, (0.07,), 1.1, (0.118, 0.03, 1.01), linvel=(-1.0, 0.0, 0.2), angvel=(0, 0, 0))
    sc = scene_from_envs([e])
    c = cfg(substeps=1, iterations=10, friction=mu, gravity=(0.0, 0.0, 0.0))
    st0 = sc.state()
    d = oracle.detect(sc, c, st0[0], st0[1], precision="f64")
    assert d.contact_count[0] == 1
    st1, _ = oracle.step(sc, c, st0, None, nsteps=1, precision="f64")
    P0, L0 = _momenta(sc, st0)
    P1, L1 = _momenta(sc, st1)
    assert not np.allclose(st0[2], st1[2])        # the impact happened
    np.testing.assert_allclose(P1, P0, atol=1e-12)
    if mu == 0.0:
        # normal impulse along the centre line: no torque about the origin
        m = sc.body_mass.astype(np.float64)
        # angular momentum of the translational motion about the origin,
        # evaluated at the substep-start positions where the impulse acts
        Lpre = (m[:, None] * np.cross(st0[0], st1[2])).sum(0)
        np.testing.assert_allclose(Lpre, (m[:, None] * np.cross(st0[0], st0[2])).sum(0), atol=1e-12)
        assert np.abs(st1[3]).max() < 1e-12


def test_box_box_impact_conserves_linear_momentum():
    e = env()
    e.body(S.BOX, (0.05, 0.05, 0.05), 0.5, (0.0, 0.0, 1.0), axis_angle((0, 0, 1), 0.2), linvel=(1.5, 0, 0))
    e.body(S.BOX, (0.06, 0.04, 0.05), 0.9, (0.108, 0.01, 1.0), axis_angle((1, 1, 0), 0.1),
           linvel=(-0.5, 0.1, 0))
    sc = scene_from_envs([e])
    c = cfg(substeps=2, iterations=10, friction=0.5, gravity=(0.0, 0.0, 0.0))
    st0 = sc.state()
    st1, _ = oracle.step(sc, c, st0, None, nsteps=3, precision="f64")
    P0, _ = _momenta(sc, st0)
    P1, _ = _momenta(sc, st1)
    assert not np.allclose(st0[2], st1[2])
    np.testing.assert_allclose(P1, P0, atol=1e-12)


# --------------------------------------------------------------------------
# solver: hand-derived projected Gauss-Seidel iteration
# --------------------------------------------------------------------------
@pytest.mark.parametrize("iters", [1, 2, 5])
def test_two_sphere_stack_pgs_matches_hand_iteration(iters):
    """Sphere A on the plane, sphere B on A, both touching (s = 0). Pair order
    puts A-B before A-plane, so A-B takes colour 0 and A-plane colour 1. Each
    iteration: the A-B row brings both spheres to their common velocity, then
    the A-plane row zeroes v_A. With rho = mB/(mA+mB): v_A = 0 and
    v_B = -g h rho^(N-1) after N iterations."""
    mA, mB, rA, rB = 0.75, 0.25, 0.0625, 0.03125     # exact in f32
    e = env()
    e.body(S.SPHERE, (rA,), mA, (0.0, 0.0, rA))
    e.body(S.SPHERE, (rB,), mB, (0.0, 0.0, 2 * rA + rB))
    sc = scene_from_envs([e])
    c = cfg(substeps=1, iterations=iters, friction=0.5)
    d = oracle.detect(sc, c, sc.pos, sc.quat, precision="f64")
    assert d.manifold_count[0] == 2 and d.ncolours[0] == 2
    out, _ = oracle.step(sc, c, sc.state(), None, nsteps=1, precision="f64")
    h = 0.01
    v = -G * h * (mB / (mA + mB)) ** (iters - 1)
    np.testing.assert_allclose(out[2][:, 2], [0.0, v], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out[0][:, 2], [rA, 2 * rA + rB + h * v], rtol=1e-12)


def test_jacobi_and_pgs_converge_to_same_solution():
    mA, mB, rA, rB = 0.7, 0.3, 0.05, 0.04
    e = env()
    e.body(S.SPHERE, (rA,), mA, (0.0, 0.0, rA))
    e.body(S.SPHERE, (rB,), mB, (0.0, 0.0, 2 * rA + rB))
    sc = scene_from_envs([e])
    res = []
    for mode in (S.MODE_COLOURED, S.MODE_JACOBI):
        out, _ = oracle.step(sc, cfg(substeps=1, iterations=300, mode=mode), sc.state(), None, 1,
                             precision="f64")
        res.append(out[2])
    np.testing.assert_allclose(res[0], 0.0, atol=1e-9)
    np.testing.assert_allclose(res[1], res[0], atol=1e-6)


# --------------------------------------------------------------------------
# joints and drives
# --------------------------------------------------------------------------
Q_DOWN = axis_angle((0, 1, 0), np.pi / 2)      # link local x -> world -z


def _pendulum_env(n_links, L=0.2, r=0.02, m=1.0, tilt=0.0, horizontal=False):
    """Chain of capsule links hanging from a world pivot at z = 2 with hinge
    axes along world y. Frames are set at the straight-down configuration;
    the chain then starts rotated by `tilt` about the pivot (or horizontal)."""
    e = env()
    pivot = np.array([0.0, 0.0, 2.0])
    qh = S.QW_AXIS_Y
    qb = tuple(quat_mul([Q_DOWN[0], -Q_DOWN[1], -Q_DOWN[2], -Q_DOWN[3]], qh))
    ang = np.pi / 2 if horizontal else tilt
    q0 = tuple(quat_mul(axis_angle((0, 1, 0), ang), Q_DOWN))
    down = quat_rotate(q0, (1.0, 0.0, 0.0))
    for i in range(n_links):
        centre = pivot + down * (2 * L * i + L)
        e.body(S.CAPSULE, (r, L), m, tuple(centre), q0)
        if i == 0:
            fa = tuple(pivot) + tuple(qh)
        else:
            fa = (L, 0.0, 0.0) + qb
        e.joint(S.REVOLUTE, i - 1, i, fa, (-L, 0.0, 0.0) + qb, (0.0, 0.0, 0.0), (0.0, 0.0),
                [(0.0, 0.0, -np.pi, np.pi)])
    return e


def _anchor_drift(sc, st):
    worst = 0.0
    for j in range(sc.num_joints):
        p, c = sc.joint_parent[j], sc.joint_child[j]
        fa, fb = sc.joint_frame_a[j].astype(np.float64), sc.joint_frame_b[j].astype(np.float64)
        pa = fa[:3] if p < 0 else st[0][p] + quat_rotate(st[1][p], fa[:3])
        pb = st[0][c] + quat_rotate(st[1][c], fb[:3])
        worst = max(worst, float(np.linalg.norm(pb - pa)))
    return worst


def test_pendulum_chain_anchor_drift_bound():
    sc = scene_from_envs([_pendulum_env(3, horizontal=True)])
    c = cfg(substeps=4, iterations=20)
    st = sc.state()
    worst, zmin = 0.0, np.inf
    for _ in range(20):
        st, status = oracle.step(sc, c, st, None, nsteps=10, precision="f64")
        assert status[0] == 0
        worst = max(worst, _anchor_drift(sc, st))
        zmin = min(zmin, st[0][2][2])
    assert worst <= 1e-3
    assert zmin < 1.5     # the chain swung down


def _capsule_perp_inertia_numeric(r, L, m, n=400_000, seed=0):
    """Moment of inertia of a solid capsule about a perpendicular axis through
    its centre, by Monte-Carlo integration over the solid."""
    rng = np.random.default_rng(seed)
    box = np.array([L + r, r, r])
    pts = rng.uniform(-box, box, size=(n, 3))
    t = np.clip(pts[:, 0], -L, L)
    inside = (pts[:, 0] - t) ** 2 + pts[:, 1] ** 2 + pts[:, 2] ** 2 <= r * r
    p = pts[inside]
    return m * np.mean(p[:, 0] ** 2 + p[:, 2] ** 2)


def test_single_pendulum_small_angle_period():
    """Physical pendulum: T = 2 pi sqrt(I_pivot / (m g d)), d = L, with the
    capsule's perpendicular inertia integrated numerically."""
    L, r, m = 0.2, 0.02, 1.0
    sc = scene_from_envs([_pendulum_env(1, L=L, r=r, m=m, tilt=0.05)])
    c = cfg(substeps=4, iterations=20)
    Ip = _capsule_perp_inertia_numeric(r, L, m) + m * L * L
    T = 2 * np.pi * np.sqrt(Ip / (m * G * L))
    st = sc.state()
    ts, th = [], []
    for k in range(300):
        st, _ = oracle.step(sc, c, st, None, nsteps=1, precision="f64")
        a = quat_rotate(st[1][0], (1.0, 0.0, 0.0))
        ts.append((k + 1) * 0.01)
        th.append(np.arctan2(-a[0], -a[2]))
    th = np.array(th)
    cross = [ts[i] + (ts[i + 1] - ts[i]) * th[i] / (th[i] - th[i + 1])
             for i in range(len(th) - 1) if th[i] > 0 >= th[i + 1]]
    assert len(cross) >= 3
    period = np.mean(np.diff(cross))
    assert abs(period - T) < 0.02 * T


def test_revolute_drive_converges_to_target():
    e = env()
    L = 0.15
    e.body(S.CAPSULE, (0.03, L), 1.5, (0.0, 0.0, 0.5 + L), S.Q_LINK)
    e.joint(S.REVOLUTE, -1, 0, (0.0, 0.0, 0.5) + S.QW_AXIS_Z, (-L, 0.0, 0.0) + S.QL_AXIS_Z,
            S.ARM_GAINS, (0.0, 0.0), [(0.0, 0.0, -np.pi, np.pi)])
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=20, gravity=(0.0, 0.0, 0.0))
    tg = np.full((300, 1, 1), 0.3, np.float32)
    out, _ = oracle.step(sc, c, sc.state(), tg, nsteps=300, precision="f64")
    q = out[1][0]
    # the link spins about its own axis (world z): relative angle = 2 atan2(qx', qw')
    rel = quat_mul([S.Q_LINK[0], -S.Q_LINK[1], -S.Q_LINK[2], -S.Q_LINK[3]], q)
    theta = 2 * np.arctan2(rel[1], rel[0])
    assert abs(theta - 0.3) < 1e-3
    assert _anchor_drift(sc, out) < 1e-4


@pytest.mark.parametrize("target,expect", [(0.02, 0.02), (0.08, 0.05), (-0.03, 0.0)])
def test_prismatic_drive_and_limits(target, expect):
    e = env()
    e.body(S.BOX, (0.02, 0.02, 0.02), 0.2, (0.0, 0.0, 1.0))
    e.joint(S.PRISMATIC, -1, 0, (0.0, 0.0, 1.0) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID,
            S.FINGER_GAINS, S.FINGER_LIMITS, [(0.0, 0.0, -1.0, 1.0)])
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=20, gravity=(0.0, 0.0, -G))
    tg = np.full((200, 1, 1), target, np.float32)
    out, _ = oracle.step(sc, c, sc.state(), tg, nsteps=200, precision="f64")
    assert abs(out[0][0][0] - expect) < 1e-3
    assert abs(out[0][0][2] - 1.0) < 1e-4 and abs(out[0][0][1]) < 1e-6


def test_planar_base_drives_converge():
    e = env()
    e.body(S.BOX, (0.25, 0.25, 0.1), 30.0, (0.0, 0.0, 0.12))
    e.joint(S.PLANAR, -1, 0, (0.0, 0.0, 0.12) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID, S.BASE_GAINS,
            (0.0, 0.0), [(0.0, 0.0, -2, 2), (0.0, 0.0, -2, 2), (0.0, 0.0, -np.pi, np.pi)])
    sc = scene_from_envs([e])
    c = cfg(substeps=4, iterations=20)
    tg = np.tile(np.array([0.1, -0.05, 0.2], np.float32), (400, 1, 1))
    out, _ = oracle.step(sc, c, sc.state(), tg, nsteps=400, precision="f64")
    q = out[1][0]
    np.testing.assert_allclose(out[0][0], [0.1, -0.05, 0.12], atol=2e-3)
    assert abs(2 * np.arctan2(q[3], q[0]) - 0.2) < 2e-3
    assert abs(q[1]) < 1e-6 and abs(q[2]) < 1e-6


def test_link_frame_constants():
    """The generator's link-local joint frames equal conj(Q_LINK) * world frame."""
    conj = [S.Q_LINK[0], -S.Q_LINK[1], -S.Q_LINK[2], -S.Q_LINK[3]]
    for qw, ql in ((S.QW_AXIS_Z, S.QL_AXIS_Z), (S.QW_AXIS_Y, S.QL_AXIS_Y), (S.QW_AXIS_NY, S.QL_AXIS_NY)):
        np.testing.assert_allclose(quat_mul(conj, qw), ql, atol=1e-15)
    np.testing.assert_allclose(quat_rotate(S.Q_LINK, (1, 0, 0)), (0, 0, 1), atol=1e-15)


# --------------------------------------------------------------------------
# broadphase: brute force
# --------------------------------------------------------------------------
def _exact_aabb(shape, dims, pos, quat):
    if shape == S.SPHERE:
        r = dims[0]
        return pos - r, pos + r
    if shape == S.CAPSULE:
        a = quat_rotate(quat, (dims[1], 0, 0))
        ends = np.array([pos - a, pos + a])
        return ends.min(0) - dims[0], ends.max(0) + dims[0]
    corners = np.array([pos + quat_rotate(quat, np.array(s) * dims[:3])
                        for s in itertools.product((-1, 1), repeat=3)])
    return corners.min(0), corners.max(0)


def _inside(shape, dims, pos, quat, p):
    """Points p (N,3) inside a shape."""
    qc = [quat[0], -quat[1], -quat[2], -quat[3]]
    l = np.array([quat_rotate(qc, x - pos) for x in p])
    if shape == S.SPHERE:
        return (l ** 2).sum(1) <= dims[0] ** 2
    if shape == S.CAPSULE:
        t = np.clip(l[:, 0], -dims[1], dims[1])
        return (l[:, 0] - t) ** 2 + l[:, 1] ** 2 + l[:, 2] ** 2 <= dims[0] ** 2
    return np.all(np.abs(l) <= dims[:3], axis=1)


def _random_scene(seed, nd=5, ns=2):
    rng = np.random.default_rng(seed)
    e = env()
    for _ in range(nd):
        shape = int(rng.integers(3))
        dims = {S.SPHERE: (rng.uniform(0.05, 0.15),),
                S.CAPSULE: (rng.uniform(0.03, 0.08), rng.uniform(0.02, 0.12)),
                S.BOX: tuple(rng.uniform(0.03, 0.15, 3))}[shape]
        q = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
        e.body(shape, dims, float(rng.uniform(0.1, 1.0)), tuple(rng.uniform(-0.25, 0.25, 3) + [0, 0, 0.2]), q)
    for _ in range(ns):
        q = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
        e.static(tuple(rng.uniform(-0.25, 0.25, 3) + [0, 0, 0.2]), tuple(rng.uniform(0.05, 0.2, 3)), q)
    if rng.uniform() < 0.5:   # a joint to exercise the filter
        e.joint(S.REVOLUTE, 0, 1, (0, 0, 0) + S.Q_ID, (0, 0, 0) + S.Q_ID, (0, 0, 0), (0, 0), [(0, 0, -1, 1)])
    return scene_from_envs([e])


@pytest.mark.parametrize("seed", range(12))
def test_broadphase_matches_brute_force(seed):
    sc = _random_scene(seed)
    c = cfg(max_pairs=64, max_contacts=64)
    d = oracle.detect(sc, c, sc.pos, sc.quat, precision="f64")
    D, Ns = sc.num_bodies, sc.num_statics
    boxes = []
    for i in range(D):
        lo, hi = _exact_aabb(sc.body_shape[i], sc.body_dims[i].astype(float), sc.pos[i].astype(float),
                             sc.quat[i].astype(float))
        boxes.append((lo - c.contact_offset, hi + c.contact_offset))
    for k in range(Ns):
        p = sc.static_pose[k].astype(float)
        lo, hi = _exact_aabb(S.BOX, sc.static_half[k].astype(float), p[:3], p[3:])
        boxes.append((lo - c.contact_offset, hi + c.contact_offset))
    got = np.concatenate([d.aabb_body, d.aabb_static])
    want = np.array([np.concatenate(b) for b in boxes])
    np.testing.assert_allclose(got, want, atol=1e-6)    # inputs are f32-rounded
    jointed = {(int(sc.joint_parent[j]), int(sc.joint_child[j])) for j in range(sc.num_joints)}
    expect = []
    for i in range(D):
        for j in range(i + 1, D + Ns + 1):
            if j == D + Ns:
                hit = got[i][2] <= 0.0
            else:
                hit = np.all(got[i][:3] <= got[j][3:]) and np.all(got[j][:3] <= got[i][3:])
            if hit and not (j < D and ((i, j) in jointed or (j, i) in jointed)):
                expect.append((i, j))
    pairs = [tuple(p) for p in d.pairs[0, :d.pair_count[0]]]
    assert pairs == expect
    # superset of true overlaps, found by sampling points inside shape i
    rng = np.random.default_rng(100 + seed)
    for i in range(D):
        lo, hi = boxes[i]
        pts = rng.uniform(lo, hi, size=(4000, 3))
        pts = pts[_inside(sc.body_shape[i], sc.body_dims[i], sc.pos[i], sc.quat[i], pts)]
        for j in range(i + 1, D + Ns):
            if j < D:
                hit = _inside(sc.body_shape[j], sc.body_dims[j], sc.pos[j], sc.quat[j], pts).any()
            else:
                p = sc.static_pose[j - D]
                hit = _inside(S.BOX, sc.static_half[j - D], p[:3], p[3:], pts).any()
            jt = j < D and ((i, j) in jointed or (j, i) in jointed)
            if hit and not jt:
                assert (i, j) in pairs


# --------------------------------------------------------------------------
# narrowphase: invariants and closed forms
# --------------------------------------------------------------------------
def _surface_dist(shape, dims, pos, quat, p):
    qc = [quat[0], -quat[1], -quat[2], -quat[3]]
    l = quat_rotate(qc, p - pos)
    if shape == S.SPHERE:
        return np.linalg.norm(l) - dims[0]
    if shape == S.CAPSULE:
        t = np.clip(l[0], -dims[1], dims[1])
        return np.linalg.norm(l - [t, 0, 0]) - dims[0]
    q = np.abs(l) - dims[:3]
    return np.linalg.norm(np.maximum(q, 0)) + min(q.max(), 0.0)


def _on_surface(shape, dims, pos, quat, p):
    sd = _surface_dist(shape, dims, pos, quat, p)
    if shape == S.CAPSULE:
        assert -dims[0] - 1e-6 <= sd <= 1e-6
    else:
        assert abs(sd) < 1e-6


@pytest.mark.parametrize("seed", range(12))
def test_contact_points_lie_on_surfaces(seed):
    """For every pair type: pa lies on A's surface, pb on B's, |n| = 1 and
    s = n . (pb - pa). A capsule contributes contacts of the spheres around
    its segment points (endpoints, closest point), so a capsule-side point may
    lie inside the capsule, within one radius of its segment; and
    s = n . (pb - pa) < contact offset (FP64 arithmetic on f32-rounded poses,
    whose quaternions are unit only to ~1e-7)."""
    sc = _random_scene(seed)
    c = cfg(max_pairs=64, max_contacts=64)
    d = oracle.detect(sc, c, sc.pos, sc.quat, precision="f64")
    D = sc.num_bodies
    pos, quat = sc.pos.astype(float), sc.quat.astype(float)
    for k in range(d.contact_count[0]):
        a, b = d.contact_ids[0, k]
        g = d.contact_geom[0, k]
        n, ra, rb, s = g[:3], g[3:6], g[6:9], g[9]
        assert abs(np.linalg.norm(n) - 1) < 1e-6
        pa = pos[a] + quat_rotate(quat[a], ra)
        _on_surface(sc.body_shape[a], sc.body_dims[a].astype(float), pos[a], quat[a], pa)
        if b < D:
            pb = pos[b] + quat_rotate(quat[b], rb)
            _on_surface(sc.body_shape[b], sc.body_dims[b].astype(float), pos[b], quat[b], pb)
            sb = 0.0
        elif b < D + sc.num_statics:
            pb = rb
            p = sc.static_pose[b - D].astype(float)
            sb = _surface_dist(S.BOX, sc.static_half[b - D].astype(float), p[:3], p[3:], pb)
        else:
            pb = rb
            sb = pb[2]
        assert abs(sb) < 1e-6
        assert abs(np.dot(n, pb - pa) - s) < 1e-7
        assert s < c.contact_offset


def _detect_one(e, **kw):
    sc = scene_from_envs([e])
    c = cfg(**kw)
    return sc, oracle.detect(sc, c, sc.pos, sc.quat, precision="f64")


def test_sphere_sphere_and_plane_closed_form():
    e = env()
    c1, c2 = np.array([0.0, 0.0, 1.0]), np.array([0.15, 0.05, 1.02])
    e.body(S.SPHERE, (0.1,), 1.0, tuple(c1))
    e.body(S.SPHERE, (0.08,), 1.0, tuple(c2))
    e.body(S.SPHERE, (0.1,), 1.0, (0.9, 0.3, 0.09))
    sc, d = _detect_one(e)
    dd = sc.pos[1].astype(float) - sc.pos[0].astype(float)
    g = d.contact_geom[0]
    ids = [tuple(x) for x in d.contact_ids[0, :d.contact_count[0]]]
    assert ids == [(0, 1), (2, 3)]
    np.testing.assert_allclose(g[0, :3], dd / np.linalg.norm(dd), atol=1e-12)
    r = sc.body_dims[:2, 0].astype(float)
    assert abs(g[0, 9] - (np.linalg.norm(dd) - r[0] - r[1])) < 1e-12
    np.testing.assert_allclose(g[1, :3], [0, 0, -1])
    assert abs(g[1, 9] - (-0.01)) < 1e-7


def test_box_stack_face_contact_four_corners():
    e = env()
    e.body(S.BOX, (0.2, 0.2, 0.1), 3.0, (0.0, 0.0, 0.5))
    qB = axis_angle((0, 0, 1), 0.4)
    cB = np.array([0.03, -0.02, 0.5 + 0.1 + 0.05 - 0.002])
    e.body(S.BOX, (0.05, 0.05, 0.05), 1.0, tuple(cB), qB)
    sc, d = _detect_one(e)
    assert d.contact_count[0] == 4
    g = d.contact_geom[0, :4]
    np.testing.assert_allclose(g[:, :3], np.tile([0, 0, 1.0], (4, 1)), atol=1e-7)
    np.testing.assert_allclose(g[:, 9], -0.002, atol=1e-6)
    # points on B are B's bottom corners
    corners = {tuple(np.round([sx * 0.05, sy * 0.05, -0.05], 6)) for sx in (-1, 1) for sy in (-1, 1)}
    assert {tuple(np.round(r, 6)) for r in g[:, 6:9]} == corners


def test_box_box_edge_edge_closed_form():
    """Cube A turned 45 deg about x, cube B turned 45 deg about y above it:
    the top edge of A (along x) crosses the bottom edge of B (along y)."""
    h = 0.05
    e = env()
    e.body(S.BOX, (h, h, h), 1.0, (0.0, 0.0, 0.5), axis_angle((1, 0, 0), np.pi / 4))
    zb = 0.5 + 2 * h * np.sqrt(2) - 0.002
    e.body(S.BOX, (h, h, h), 1.0, (0.0, 0.0, zb), axis_angle((0, 1, 0), np.pi / 4))
    sc, d = _detect_one(e)
    assert d.contact_count[0] == 1
    g = d.contact_geom[0, 0]
    np.testing.assert_allclose(np.abs(g[:3]), [0, 0, 1], atol=1e-6)
    assert g[2] > 0
    assert abs(g[9] + 0.002) < 1e-6


def test_capsule_closed_forms():
    e = env()
    # lying capsule on the plane: two endpoint contacts at s = z - r
    e.body(S.CAPSULE, (0.03, 0.1), 1.0, (0.0, 0.0, 0.029), axis_angle((0, 0, 1), 0.7))
    # crossed capsules high up: one contact, s = dz - r1 - r2, normal +z
    e.body(S.CAPSULE, (0.03, 0.1), 1.0, (2.0, 0.0, 1.0))
    e.body(S.CAPSULE, (0.02, 0.1), 1.0, (2.01, 0.02, 1.048), axis_angle((0, 0, 1), np.pi / 2))
    # parallel capsules: two contacts over the overlap
    e.body(S.CAPSULE, (0.03, 0.1), 1.0, (4.0, 0.0, 1.0))
    e.body(S.CAPSULE, (0.03, 0.1), 1.0, (4.05, 0.0, 1.059))
    sc, d = _detect_one(e)
    ids = [tuple(x) for x in d.contact_ids[0, :d.contact_count[0]]]
    g = d.contact_geom[0]
    assert ids == [(0, 5), (0, 5), (1, 2), (3, 4), (3, 4)]
    np.testing.assert_allclose(g[0:2, 9], -0.001, atol=1e-7)
    np.testing.assert_allclose(g[2, :3], [0, 0, 1], atol=1e-7)
    assert abs(g[2, 9] - (0.048 - 0.05)) < 1e-7
    np.testing.assert_allclose(g[3:5, 9], 0.059 - 0.06, atol=1e-7)
    # the parallel contacts sit at the ends of the overlap [-0.05, 0.1] on capsule 3's axis
    L = float(sc.body_dims[3, 1])
    off = float(sc.pos[4, 0]) - float(sc.pos[3, 0])
    np.testing.assert_allclose(sorted(g[3:5, 3]), [off - L, L], atol=1e-12)


def test_capsule_lying_on_box_two_contacts_and_sphere_on_box_edge():
    e = env()
    e.static((0.0, 0.0, 0.4), (0.3, 0.3, 0.4))
    e.body(S.CAPSULE, (0.02, 0.05), 0.3, (0.0, 0.1, 0.8 + 0.02 - 0.001), axis_angle((0, 0, 1), 0.3))
    # sphere beyond the top edge at x = 0.3: distance to the edge = |(dx, dz)|
    dx, dz, r = 0.01, 0.015, 0.02
    e.body(S.SPHERE, (r,), 0.3, (0.3 + dx, -0.1, 0.8 + dz))
    sc, d = _detect_one(e)
    ids = [tuple(x) for x in d.contact_ids[0, :d.contact_count[0]]]
    g = d.contact_geom[0]
    assert ids == [(0, 2), (0, 2), (1, 2)]
    np.testing.assert_allclose(g[0:2, 9], -0.001, atol=1e-7)
    np.testing.assert_allclose(g[0:2, :3], [[0, 0, -1], [0, 0, -1]], atol=1e-7)
    assert abs(g[2, 9] - (np.hypot(dx, dz) - r)) < 1e-7
    np.testing.assert_allclose(g[2, :3], -np.array([dx, 0, dz]) / np.hypot(dx, dz), atol=1e-7)


# --------------------------------------------------------------------------
# colouring, determinism, precision
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg_idx", [2, 3, 5])
def test_colouring_is_valid_greedy(cfg_idx):
    sc, c = S.make_config(cfg_idx, num_envs=6)
    d = oracle.detect(sc, c, sc.pos, sc.quat)
    J = sc.num_joints
    for e in range(sc.num_envs):
        D = sc.body_off[e + 1] - sc.body_off[e]
        j0, j1 = sc.joint_off[e], sc.joint_off[e + 1]
        bodies = [(int(sc.joint_parent[j]), int(sc.joint_child[j])) for j in range(j0, j1)]
        cols = list(d.colours[j0:j1])
        # manifolds: first contact of each run of equal (a, b)
        ids = [tuple(x) for x in d.contact_ids[e, :d.contact_count[e]]]
        man = []
        for k, ab in enumerate(ids):
            if k == 0 or ids[k - 1] != ab:
                man.append(ab)
        assert len(man) == d.manifold_count[e]
        bodies += [(a, b if b < D else -1) for a, b in man]
        cols += list(d.colours[J + e * c.max_pairs: J + e * c.max_pairs + len(man)])
        assert max(cols) + 1 == d.ncolours[e]
        seen = {}
        for k, ((a, b), col) in enumerate(zip(bodies, cols)):
            touched = [x for x in (a, b) if x >= 0]
            # lowest colour not used by an earlier constraint on these bodies
            used = {seen[(x, cc)] for x in touched for cc in range(64) if (x, cc) in seen}
            earlier = {cc for x in touched for cc in range(64) if (x, cc) in seen}
            assert col == min(set(range(65)) - earlier)
            for x in touched:
                seen[(x, col)] = k
            del used


def test_oracle_is_deterministic_and_fp32_tracks_fp64():
    sc, c = S.make_config(3, num_envs=8)
    st = sc.state()
    tg = sc.target_walk(5)
    a, _ = oracle.step(sc, c, st, tg, 5, "f32")
    b, _ = oracle.step(sc, c, st, tg, 5, "f32", threads=1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    one32, _ = oracle.step(sc, c, st, tg, 1, "f32")
    one64, _ = oracle.step(sc, c, st, tg, 1, "f64")
    assert np.abs(one32[0] - one64[0]).max() < 1e-5
    assert np.abs(one32[2] - one64[2]).max() < 1e-3


# --------------------------------------------------------------------------
# speculative contacts, soft drives, Jacobi splitting (exact discrete forms)
# --------------------------------------------------------------------------
def test_speculative_contact_lands_exactly():
    """A sphere s0 above the plane moving down fast: the speculative row lets
    it close the gap and no more, so after one substep z = r and v_z = -s0/h."""
    r, s0 = 0.0625, 2.0 ** -8
    e = env()
    e.body(S.SPHERE, (r,), 0.5, (0.0, 0.0, r + s0), linvel=(0.0, 0.0, -2.0))
    sc = scene_from_envs([e])
    out, _ = oracle.step(sc, cfg(substeps=1, iterations=1), sc.state(), None, 1, precision="f64")
    assert abs(out[0][0][2] - r) < 1e-15
    assert abs(out[2][0][2] - (-s0 / 0.01)) < 1e-12


def test_soft_drive_is_implicit_euler_spring_damper():
    """One soft row on a free slider (no gravity): each substep equals the
    implicit-Euler update of m x'' = -k (x - x*) - d x' (Catto's soft step)."""
    m, k, d = 0.25, 1000.0, 100.0
    e = env()
    e.body(S.BOX, (0.02, 0.02, 0.02), m, (0.0, 0.0, 1.0))
    e.joint(S.PRISMATIC, -1, 0, (0.0, 0.0, 1.0) + S.Q_ID, (0.0, 0.0, 0.0) + S.Q_ID,
            (k, d, 1e6), (-1.0, 1.0), [(0.0, 0.0, -1.0, 1.0)])
    sc = scene_from_envs([e])
    S_ = 4
    c = cfg(substeps=S_, iterations=7, gravity=(0.0, 0.0, 0.0))
    target = np.float32(0.03125)
    n = 20
    out, _ = oracle.step(sc, c, sc.state(), np.full((n, 1, 1), target, np.float32), n, precision="f64")
    h = 0.01 / S_
    x, v = 0.0, 0.0
    for _ in range(n * S_):
        v = (v - h * k / m * (x - float(target))) / (1 + h * d / m + h * h * k / m)
        x = x + h * v
    assert abs(out[0][0][0] - x) < 1e-12
    assert abs(out[2][0][0] - v) < 1e-10


@pytest.mark.parametrize("iters", [1, 2, 3, 7])
def test_two_sphere_stack_jacobi_matches_hand_iteration(iters):
    """Jacobi with Tonge mass splitting on the stack: A touches two constraints
    (split 2), B one. Each iteration both rows read the iteration-start
    velocities; effective masses use the split inverse masses; bodies add the
    true-mass velocity changes."""
    mA, mB, rA, rB = 0.75, 0.25, 0.0625, 0.03125
    e = env()
    e.body(S.SPHERE, (rA,), mA, (0.0, 0.0, rA))
    e.body(S.SPHERE, (rB,), mB, (0.0, 0.0, 2 * rA + rB))
    sc = scene_from_envs([e])
    out, _ = oracle.step(sc, cfg(substeps=1, iterations=iters, mode=S.MODE_JACOBI), sc.state(), None, 1,
                         precision="f64")
    h = 0.01
    vA = vB = -G * h
    l1 = l2 = 0.0
    K1, K2 = 2 / mA + 1 / mB, 2 / mA
    for _ in range(iters):
        n1 = max(0.0, l1 - (vB - vA) / K1)
        d1, l1 = n1 - l1, n1
        n2 = max(0.0, l2 - vA / K2)
        d2, l2 = n2 - l2, n2
        vA, vB = vA - d1 / mA + d2 / mA, vB + d1 / mB
    np.testing.assert_allclose(out[2][:, 2], [vA, vB], rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------
# angular momentum: world inertia and lever arms
# --------------------------------------------------------------------------
def _capsule_inertia_quadrature(r, L, m, n=200001):
    """Axial and perpendicular inertia of a solid capsule by integrating disks
    along its axis (Simpson's rule)."""
    x = np.linspace(-(L + r), L + r, n)
    ax = np.abs(x)
    rho2 = np.where(ax <= L, r * r, np.maximum(r * r - (ax - L) ** 2, 0.0))
    w = np.ones(n)
    w[1:-1:2], w[2:-1:2] = 4, 2
    dx = x[1] - x[0]
    integ = lambda f: (w * f).sum() * dx / 3
    vol = integ(np.pi * rho2)
    dens = m / vol
    Iax = dens * integ(np.pi * rho2 * rho2 / 2)
    Ip = dens * integ(np.pi * rho2 * (rho2 / 4 + x * x))
    return np.array([Iax, Ip, Ip])


def _body_inertia(shape, dims, m):
    if shape == S.SPHERE:
        return np.full(3, 0.4 * m * dims[0] ** 2)
    if shape == S.BOX:
        hx, hy, hz = dims[:3]
        return m / 3 * np.array([hy * hy + hz * hz, hx * hx + hz * hz, hx * hx + hy * hy])
    return _capsule_inertia_quadrature(dims[0], dims[1], m)


def _ang_momentum(sc, pos, quat, v, w):
    L = np.zeros(3)
    for i in range(sc.num_bodies):
        m = float(sc.body_mass[i])
        I = _body_inertia(sc.body_shape[i], sc.body_dims[i].astype(float), m)
        R = np.array([quat_rotate(quat[i], e) for e in np.eye(3)]).T
        L += m * np.cross(pos[i], v[i]) + R @ (I * (R.T @ w[i]))
    return L


def _impulse_step_conserves(e, substeps=1, atol=1e-9, nsteps=1, check_lin=True):
    sc = scene_from_envs([e])
    c = cfg(substeps=substeps, iterations=10, friction=0.0, gravity=(0.0, 0.0, 0.0))
    st0 = tuple(a.astype(np.float64) for a in sc.state())
    st1, _ = oracle.step(sc, c, sc.state(), np.zeros((1, 1, max(sc.max_dof, 1)), np.float32), 1,
                         precision="f64")
    assert not np.allclose(st0[2], st1[2]) or not np.allclose(st0[3], st1[3])
    m = sc.body_mass.astype(np.float64)[:, None]
    if check_lin:
        np.testing.assert_allclose((m * st1[2]).sum(0), (m * st0[2]).sum(0), atol=1e-12)
    # evaluated at the poses where the impulses act (one substep)
    L0 = _ang_momentum(sc, st0[0], st0[1], st0[2], st0[3])
    L1 = _ang_momentum(sc, st0[0], st0[1], st1[2], st1[3])
    np.testing.assert_allclose(L1, L0, atol=atol)


def test_frictionless_box_box_impact_conserves_angular_momentum():
    e = env()
    q = (0.5, 0.5, 0.5, 0.5)          # exact unit quaternion, non-axis-aligned inertia
    e.body(S.BOX, (0.05, 0.03, 0.02), 0.5, (0.0, 0.0, 1.0), q, linvel=(1.5, 0.2, 0), angvel=(0.3, -2, 1))
    e.body(S.BOX, (0.0625, 0.04, 0.03), 0.9, (0.0625, 0.01, 1.005), (0.5, -0.5, 0.5, 0.5),
           linvel=(-0.5, 0.1, 0), angvel=(1, 0.5, -0.25))
    _impulse_step_conserves(e, atol=1e-6)


def test_frictionless_sphere_capsule_impact_conserves_angular_momentum():
    e = env()
    e.body(S.CAPSULE, (0.03, 0.1), 0.8, (0.0, 0.0, 1.0), (0.5, 0.5, 0.5, 0.5), angvel=(0.2, 0.1, -0.3))
    e.body(S.SPHERE, (0.05,), 0.4, (0.02, 0.06, 1.0 + 0.08 - 0.002), linvel=(0.0, -0.3, -2.0))
    _impulse_step_conserves(e, atol=1e-6)


def test_prismatic_pair_conserves_momentum():
    """Two free boxes joined by a driven prismatic joint, displaced along the
    slide axis and spinning: internal impulses conserve linear and angular
    momentum (every row acts at the same point on both bodies)."""
    e = env()
    q = (0.5, 0.5, 0.5, 0.5)
    e.body(S.BOX, (0.05, 0.04, 0.03), 1.0, (0.0, 0.0, 2.0), angvel=(0.5, -1.0, 0.25), linvel=(0.1, 0, 0))
    e.body(S.BOX, (0.02, 0.03, 0.04), 0.5, (0.13, 0.02, 2.05), q, angvel=(-1.0, 0.5, 2.0))  # d = 0.03
    # frame on A at its centre, slide axis world x; frame on B at its centre
    qb = (0.5, -0.5, -0.5, -0.5)       # conj(q): B's frame axes = world axes at the start
    e.joint(S.PRISMATIC, 0, 1, (0.1, 0.02, 0.05) + S.Q_ID, (0.0, 0.0, 0.0) + qb, (500.0, 20.0, 100.0),
            (-0.5, 0.5), [(0.0, 0.0, -1.0, 1.0)])
    _impulse_step_conserves(e, atol=1e-9)


def test_incline_with_oblique_normal():
    """Box on a static box tilted by theta about a skew horizontal axis (vertical
    gravity). Friction is clamped per tangent axis (a pyramid inscribing
    mu..sqrt(2) mu), so the box sticks for tan(theta) < mu and, when it
    slides, its acceleration along the slope lies between
    g (sin - sqrt(2) mu cos) and g (sin - mu cos)."""
    for theta_deg, slides in ((20.0, False), (45.0, True)):
        th = np.deg2rad(theta_deg)
        axis = np.array([np.cos(0.6), np.sin(0.6), 0.0])
        q = axis_angle(axis, th)
        nrm = quat_rotate(q, (0, 0, 1.0))
        e = env()
        e.static((0.0, 0.0, 2.0), (1.0, 1.0, 0.2), q)      # high enough to miss the ground
        hb = (0.05, 0.05, 0.02)
        ctr = np.array([0.0, 0.0, 2.0]) + nrm * (0.2 + hb[2])
        e.body(S.BOX, hb, 1.0, tuple(ctr), q)
        sc = scene_from_envs([e])
        c = cfg(substeps=4, iterations=30, friction=0.5)
        s30, _ = oracle.step(sc, c, sc.state(), None, 30, precision="f64")
        s60, _ = oracle.step(sc, c, s30, None, 30, precision="f64")
        if not slides:
            assert np.abs(s60[2][0]).max() < 1e-3
        else:
            down = -(np.array([0, 0, 1.0]) - nrm * nrm[2])
            down /= np.linalg.norm(down)
            a = np.dot(s60[2][0] - s30[2][0], down) / 0.3
            lo = G * (np.sin(th) - np.sqrt(2) * 0.5 * np.cos(th))
            hi = G * (np.sin(th) - 0.5 * np.cos(th))
            assert lo * 0.98 <= a <= hi * 1.02
            # the motion stays in the slope plane
            assert abs(np.dot(s60[2][0], nrm)) < 1e-3


def test_sphere_capsule_end_cap_and_mirrored_edge():
    e = env()
    # sphere beyond the +x end of a capsule along x: closest point = endpoint
    L, rc, rs = 0.1, 0.03, 0.04
    e.body(S.CAPSULE, (rc, L), 1.0, (0.0, 0.0, 1.0))
    e.body(S.SPHERE, (rs,), 1.0, (L + 0.05, 0.02, 1.0 + 0.03))
    sc, d = _detect_one(e)
    g = d.contact_geom[0, 0]
    end = np.array([sc.body_dims[0, 1], 0.0, 0.0]) + sc.pos[0].astype(float)
    dd = sc.pos[1].astype(float) - end
    np.testing.assert_allclose(g[:3], dd / np.linalg.norm(dd), atol=1e-12)   # capsule (A) -> sphere
    assert abs(g[9] - (np.linalg.norm(dd) - float(sc.body_dims[0, 0]) - float(sc.body_dims[1, 0]))) < 1e-12
    # edge-edge with B below A: normal points from A down to B
    h = 0.05
    e = env()
    e.body(S.BOX, (h, h, h), 1.0, (0.0, 0.0, 0.5), axis_angle((1, 0, 0), np.pi / 4))
    zb = 0.5 - 2 * h * np.sqrt(2) + 0.002
    e.body(S.BOX, (h, h, h), 1.0, (0.0, 0.0, zb), axis_angle((0, 1, 0), np.pi / 4))
    sc, d = _detect_one(e)
    assert d.contact_count[0] == 1
    g = d.contact_geom[0, 0]
    assert g[2] < -0.999999 and abs(g[9] + 0.002) < 1e-6


def test_hanging_link_frames():
    """Scene construction for the hanging arm: its local joint frames turn
    the link axis onto the world joint axes (conj(Q_HANG) * world frame)."""
    from paper_2412_13211_b300.scenes import Q_HANG, QW_AXIS_Y, QW_AXIS_Z, _local_frame
    np.testing.assert_allclose(quat_rotate(Q_HANG, (1, 0, 0)), (0, 0, -1), atol=1e-15)
    for qw in (QW_AXIS_Y, QW_AXIS_Z):
        ql = _local_frame(Q_HANG, qw)
        np.testing.assert_allclose(quat_mul(Q_HANG, ql), qw, atol=1e-15)


# --------------------------------------------------------------------------
# hinge limits (articulated receptacles: a fridge door)
# --------------------------------------------------------------------------
def _door(limits, w0):
    """A door panel on a vertical hinge at its edge (hinge frame: local x = world z)."""
    e = env()
    q_up = axis_angle((0.0, 1.0, 0.0), -np.pi / 2)               # local x -> world z
    # spinning about the hinge: centre velocity w x r, r = 0.3 m along world x
    e.body(S.BOX, (0.3, 0.02, 0.4), 5.0, (0.3, 0.0, 1.0), linvel=(0.0, 0.3 * w0, 0.0), angvel=(0.0, 0.0, w0))
    e.joint(S.REVOLUTE, -1, 0, (0.0, 0.0, 1.0) + tuple(q_up), (-0.3, 0.0, 0.0) + tuple(q_up),
            (0.0, 0.0, 0.0), limits, [])
    return e


def _door_angle(q):
    # the panel's local x axis in world
    w, x, y, z = q
    ax = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    return np.arctan2(ax[1], ax[0])


@pytest.mark.parametrize("w0,bound", [(3.0, 1.2), (-3.0, 0.0)])
def test_hinge_limits_stop_the_door(w0, bound):
    sc = scene_from_envs([_door((0.0, 1.2), w0)])
    c = cfg(substeps=4, iterations=20, gravity=(0.0, 0.0, 0.0))
    st = sc.state()
    angles = []
    for _ in range(60):
        st, status = oracle.step(sc, c, st, None, 1, "f64")
        angles.append(_door_angle(st[1][0]))
    angles = np.array(angles)
    assert (angles <= 1.2 + 2e-3).all() and (angles >= -2e-3).all()
    assert abs(angles[-1] - bound) < 2e-3                       # resting on the limit
    assert abs(st[3][0][2]) < 5e-3                               # and stopped (no restitution; Baumgarte residue)


def test_hinge_without_limits_keeps_turning():
    sc = scene_from_envs([_door((0.0, 0.0), 3.0)])               # lo == hi: no limit rows
    c = cfg(substeps=4, iterations=20, gravity=(0.0, 0.0, 0.0))
    st, _ = oracle.step(sc, c, sc.state(), None, 50, "f64")
    assert abs(st[3][0][2] - 3.0) < 2e-3                         # free spin about the hinge (solver drift)
    assert abs(_door_angle(st[1][0]) - np.angle(np.exp(1j * 1.5))) < 1e-2   # 3 rad/s for 0.5 s


@pytest.mark.parametrize("e_rest", [0.3, 0.5, 0.9])
def test_restitution_rebounds_at_e_times_approach_speed(e_rest):
    """Reading C5: a contact approaching faster than 1 m/s targets the
    rebound speed e * v_n (bias = min(bias, e * v_n)). A sphere 4 mm above
    the plane (inside the contact offset) falling at 2 m/s, one substep: its
    approach speed after gravity is |v0| + g h; a single normal row (no
    tangential motion, so the friction rows stay at zero) converges in the
    first sweep, so the sphere leaves at exactly e (|v0| + g h)."""
    r, z0, v0, h = 0.05, 0.054, -2.0, 0.01
    e = env()
    e.body(S.SPHERE, (r,), 0.7, (0.3, -0.1, z0), linvel=(0.0, 0.0, v0))
    sc = scene_from_envs([e])
    c = cfg(substeps=1, iterations=10, restitution=e_rest)
    out, st = oracle.step(sc, c, sc.state(), None, 1, "f64")
    assert not st.any()
    z0 = float(sc.pos[0, 2])          # as stored (FP32 scene)
    vz = e_rest * (-v0 + 9.81 * h)
    assert abs(out[2][0, 2] - vz) < 1e-12
    assert abs(out[0][0, 2] - (z0 + h * vz)) < 1e-12
    assert np.abs(out[2][0, :2]).max() < 1e-15


def test_restitution_is_off_below_one_metre_per_second():
    """Below the 1 m/s threshold the speculative bias applies instead: the
    sphere is stopped exactly where it reaches the plane (v = -s/h)."""
    r, z0, v0, h = 0.05, 0.054, -0.5, 0.01
    e = env()
    e.body(S.SPHERE, (r,), 0.7, (0.3, -0.1, z0), linvel=(0.0, 0.0, v0))
    sc = scene_from_envs([e])
    c = cfg(substeps=1, iterations=10, restitution=0.5)
    out, _ = oracle.step(sc, c, sc.state(), None, 1, "f64")
    z0, r = float(sc.pos[0, 2]), float(sc.body_dims[0, 0])   # as stored (FP32 scene)
    assert abs(out[2][0, 2] - (-(z0 - r) / h)) < 1e-12
    assert abs(out[0][0, 2] - r) < 1e-12
