"""Pins of the oracle's general narrowphase manifolds against brute force.

For random poses (FP64 oracle on the stored FP32 poses):
- capsule-capsule (non-parallel axes): the separation is the distance of the
  two segments (minimised over a dense grid, then polished) minus the radii,
  along the direction between the closest points;
- capsule-box (segment outside the box): the smallest separation over the
  manifold is the segment-box distance (minimised the same way) minus the
  radius, and each end cap within the contact offset contributes its own
  sphere-box contact;
- box-box face contact: the manifold's points are vertices of the overlap
  of the incident face with the reference face, built here as the convex
  polygon of the incident face's vertices inside the reference face, the
  reference face's corners inside the incident face, and the crossings of
  their edges; with more than four such points below the contact offset, the
  chosen ones are the deepest, the farthest from it, the one spanning the
  largest triangle with those two, and the one farthest on the other side;
- box-box edge contact: the two points are the closest points of the two
  crossing edges, found by brute force over all 144 edge pairs.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

import oracle
from paper_2412_13211_b300 import scenes as S
from helpers import axis_angle, cfg, env, scene_from_envs

OFF = 0.01
# FP64 arithmetic on FP32-stored poses: a stored quaternion is unit only to
# ~1e-7, so a point taken into a box's frame and back (the reference-face
# frame, an anchor in a body frame) moves by ~1e-7 of the box's size.
TOL_FRAME = 2e-7


def _rot(q):
    """Rotation matrix of a (w, x, y, z) quaternion, R = I + 2w[u]x + 2[u]x^2
    (the quaternion is used as stored, not renormalised)."""
    w, x, y, z = (float(v) for v in q)
    U = np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])
    return np.eye(3) + 2.0 * w * U + 2.0 * U @ U


def _quat_from_x(a):
    """A unit quaternion turning the x axis onto the unit vector a."""
    x = np.array([1.0, 0.0, 0.0])
    c = float(x @ a)
    if c < -0.999999:
        return (0.0, 0.0, 0.0, 1.0)
    v = np.cross(x, a)
    q = np.array([1.0 + c, *v])
    q /= np.linalg.norm(q)
    return tuple(q)


def _detect(sc):
    return oracle.detect(sc, cfg(max_pairs=16, max_contacts=32), sc.pos, sc.quat, precision="f64")


def _pose(sc, i):
    return sc.pos[i].astype(np.float64), _rot(sc.quat[i])


def _seg_seg(p1, a1, L1, p2, a2, L2):
    """Closest points of two segments c + a t, |t| <= L: grid, then polish."""
    ts = np.linspace(-L1, L1, 241)
    us = np.linspace(-L2, L2, 241)
    diff = (p1 + a1 * ts[:, None, None]) - (p2 + a2 * us[None, :, None])
    d2 = (diff ** 2).sum(-1)
    i, j = np.unravel_index(np.argmin(d2), d2.shape)

    def f(x):
        return float(((p1 + a1 * x[0]) - (p2 + a2 * x[1])) @ ((p1 + a1 * x[0]) - (p2 + a2 * x[1])))
    r = minimize(f, [ts[i], us[j]], bounds=[(-L1, L1), (-L2, L2)], method="L-BFGS-B",
                 options=dict(ftol=1e-16, gtol=1e-14, maxiter=500))
    t, u = r.x
    return p1 + a1 * t, p2 + a2 * u, t, u


def _point_box(p, c, R, h):
    """Signed distance of a point to a box (negative inside) and the box point."""
    l = R.T @ (p - c)
    q = np.clip(l, -h, h)
    out = np.linalg.norm(l - q)
    if out > 0:
        return out, c + R @ q
    k = int(np.argmin(h - np.abs(l)))
    q = l.copy()
    q[k] = np.sign(l[k]) * h[k] if l[k] != 0 else h[k]
    return -(h[k] - abs(l[k])), c + R @ q


@pytest.mark.parametrize("seed", range(10))
def test_capsule_capsule_separation_is_segment_distance(seed):
    rng = np.random.default_rng(seed)
    r1, r2 = rng.uniform(0.02, 0.06, 2)
    L1, L2 = rng.uniform(0.03, 0.12, 2)
    q1 = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    q2 = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    a1, a2 = _rot(q1)[:, 0], _rot(q2)[:, 0]
    if np.linalg.norm(np.cross(a1, a2)) ** 2 < 1e-2:
        pytest.skip("nearly parallel axes (the two-point case has its closed-form pin)")
    c1 = np.array([0.0, 0.0, 1.0])
    # place capsule 2 so that the segments come within r1 + r2 +- 5 mm
    t, u = rng.uniform(-0.8, 0.8) * L1, rng.uniform(-0.8, 0.8) * L2
    nrm = np.cross(a1, a2)
    nrm /= np.linalg.norm(nrm)
    gap = r1 + r2 + rng.uniform(-0.005, 0.005)
    c2 = c1 + a1 * t + nrm * gap - a2 * u
    e = env()
    e.body(S.CAPSULE, (r1, L1), 1.0, tuple(c1), q1)
    e.body(S.CAPSULE, (r2, L2), 1.0, tuple(c2), q2)
    sc = scene_from_envs([e])
    d = _detect(sc)
    (x1, R1), (x2, R2) = _pose(sc, 0), _pose(sc, 1)
    rr1, rr2 = float(sc.body_dims[0, 0]), float(sc.body_dims[1, 0])
    p1, p2, _, _ = _seg_seg(x1, R1[:, 0], float(sc.body_dims[0, 1]), x2, R2[:, 0], float(sc.body_dims[1, 1]))
    dist = np.linalg.norm(p2 - p1)
    want_s = dist - rr1 - rr2
    ids = [tuple(v) for v in d.contact_ids[0, :d.contact_count[0]]]
    if want_s >= OFF:
        assert (0, 1) not in ids
        return
    assert ids.count((0, 1)) == 1
    g = d.contact_geom[0, ids.index((0, 1))]
    assert abs(g[9] - want_s) < 1e-8
    np.testing.assert_allclose(g[:3], (p2 - p1) / dist, atol=1e-5)
    pa = x1 + R1 @ g[3:6]
    np.testing.assert_allclose(pa, p1 + rr1 * g[:3], atol=1e-6)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("static", [False, True])
def test_capsule_box_separation_is_segment_box_distance(seed, static):
    rng = np.random.default_rng(100 + seed)
    hb = rng.uniform(0.05, 0.2, 3)
    qb = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    cb = np.array([0.0, 0.0, 1.0])
    r, L = rng.uniform(0.02, 0.05), rng.uniform(0.03, 0.12)
    qc = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    Rb = _rot(qb)
    # a point just outside a random face, then the capsule placed so that its
    # segment passes near it (outside the box)
    k = int(rng.integers(3))
    sg = rng.choice([-1.0, 1.0])
    loc = rng.uniform(-0.7, 0.7, 3) * hb
    loc[k] = sg * hb[k]
    nloc = np.zeros(3)
    nloc[k] = sg
    near = cb + Rb @ (loc + nloc * (r + rng.uniform(-0.004, 0.006)))
    # the capsule's axis runs nearly along the face, tilted away from it
    dl = rng.normal(size=3)
    dl[k] = 0.0
    dl /= np.linalg.norm(dl)
    dl[k] = sg * rng.uniform(0.0, 0.3)
    ac = Rb @ (dl / np.linalg.norm(dl))
    qc = _quat_from_x(ac)
    tpos = rng.uniform(-L, L) * 0.5
    cc = near - ac * tpos
    e = env()
    e.body(S.CAPSULE, (r, L), 0.5, tuple(cc), qc)
    if static:
        e.static(tuple(cb), tuple(hb), qb)
    else:
        e.body(S.BOX, tuple(hb), 1.0, tuple(cb), qb)
    sc = scene_from_envs([e])
    d = _detect(sc)
    xc, Rc = _pose(sc, 0)
    rad, Lc = float(sc.body_dims[0, 0]), float(sc.body_dims[0, 1])
    if static:
        pst = sc.static_pose[0].astype(np.float64)
        xb, Rbs, hbs = pst[:3], _rot(pst[3:]), sc.static_half[0].astype(np.float64)
    else:
        xb, Rbs = _pose(sc, 1)
        hbs = sc.body_dims[1, :3].astype(np.float64)
    a = Rc[:, 0]

    def dist(t):
        return _point_box(xc + a * t, xb, Rbs, hbs)[0]
    ts = np.linspace(-Lc, Lc, 4001)
    dv = np.array([dist(t) for t in ts])
    if dv.min() <= 0:
        pytest.skip("segment touches the box (the manifold then follows the penetrating cap)")
    i = int(np.argmin(dv))
    res = minimize_scalar(dist, bounds=(ts[max(i - 1, 0)], ts[min(i + 1, len(ts) - 1)]), method="bounded",
                          options=dict(xatol=1e-12))
    tmin, dmin = float(res.x), float(res.fun)
    cnt = d.contact_count[0]
    seps = d.contact_geom[0, :cnt, 9]
    want = dmin - rad
    ends = [dist(-Lc) - rad, dist(Lc) - rad]
    if min(want, *ends) >= OFF:
        assert cnt == 0
        return
    assert cnt >= 1
    # the interior minimiser is a contact unless it lies within 1 mm of an end
    if Lc - abs(tmin) > 1e-3 + 1e-6:
        assert abs(seps.min() - want) < 1e-8, (seps, want)
    elif Lc - abs(tmin) < 1e-3 - 1e-6:
        assert abs(seps.min() - min(ends)) < 1e-8
    for s_end in ends:   # each end cap within the offset has its own contact
        if s_end < OFF:
            assert np.min(np.abs(seps - s_end)) < 1e-8


def _corners(c, R, h):
    return np.array([c + R @ (np.array(s) * h) for s in itertools.product((-1, 1), repeat=3)])


def _cross2(a, b):
    return a[0] * b[1] - a[1] * b[0]


def _overlap_polygon(P, Q):
    """Vertices of the intersection of two convex polygons in the plane (no
    clipping pass: points of each inside the other plus edge crossings)."""
    def inside(poly, x):
        n = len(poly)
        sgn = [_cross2(poly[(i + 1) % n] - poly[i], x - poly[i]) for i in range(n)]
        return all(s >= -1e-12 for s in sgn) or all(s <= 1e-12 for s in sgn)
    pts = [p for p in P if inside(Q, p)] + [q for q in Q if inside(P, q)]
    for i in range(len(P)):
        a, b = P[i], P[(i + 1) % len(P)]
        for j in range(len(Q)):
            c, dd = Q[j], Q[(j + 1) % len(Q)]
            den = _cross2(b - a, dd - c)
            if abs(den) < 1e-15:
                continue
            t = _cross2(c - a, dd - c) / den
            u = _cross2(c - a, b - a) / den
            if -1e-12 <= t <= 1 + 1e-12 and -1e-12 <= u <= 1 + 1e-12:
                pts.append(a + t * (b - a))
    out = []
    for p in pts:   # unique
        if all(np.linalg.norm(p - o) > 1e-9 for o in out):
            out.append(p)
    return out


@pytest.mark.parametrize("seed", range(24))
def test_box_box_face_manifold_is_the_reduced_face_overlap(seed):
    rng = np.random.default_rng(200 + seed)
    hA = np.array([rng.uniform(0.12, 0.2), rng.uniform(0.12, 0.2), 0.05])
    hB = np.array(rng.uniform(0.03, 0.08, 3))
    e = env()
    e.static((0.0, 0.0, 0.5), tuple(hA), axis_angle((0, 0, 1), rng.uniform(0, np.pi)))
    # tilted enough that A's face separates less than B's (A is the reference)
    ax = rng.normal(size=3)
    ax[2] = 0.0
    tilt = axis_angle(ax, rng.uniform(0.02, 0.06))
    yaw = axis_angle((0, 0, 1), rng.uniform(0, np.pi))
    w0, x0, y0, z0 = tilt
    w1, x1, y1, z1 = yaw
    qB = (w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1, w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
          w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1, w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1)
    # B hangs over A's top face (partly over an edge, so that clipping matters)
    xy = rng.uniform(-1.0, 1.0, 2) * (hA[:2] * 0.9)
    RB = _rot(qB)
    low = np.min((RB @ (np.array(list(itertools.product((-1, 1), repeat=3))) * hB).T)[2])
    zB = 0.55 - low - rng.uniform(0.0005, 0.004)
    e.body(S.BOX, tuple(hB), 1.0, (xy[0], xy[1], zB), qB)
    sc = scene_from_envs([e])
    d = _detect(sc)
    cnt = d.contact_count[0]
    # X: the dynamic box (first of the pair), Y: the static one
    xb, Rb = _pose(sc, 0)
    hb = sc.body_dims[0, :3].astype(np.float64)
    pst = sc.static_pose[0].astype(np.float64)
    xa, Ra, ha = pst[:3], _rot(pst[3:]), sc.static_half[0].astype(np.float64)
    boxes = [(xb, Rb, hb), (xa, Ra, ha)]
    # reference face: the face normal of least penetration, measured by
    # projecting the other box's corners (X's faces first, ties to X)
    best = None
    for z in (0, 1):
        cz, Rz, hz = boxes[z]
        co, Ro, ho = boxes[1 - z]
        corners = _corners(co, Ro, ho)
        for k in range(3):
            n = Rz[:, k] * (1.0 if (co - cz) @ Rz[:, k] >= 0 else -1.0)
            sep = (corners - (cz + n * hz[k])) @ n
            sep = float(sep.min())
            if best is None or sep > best[0]:
                best = (sep, z, k, n)
    # an edge-edge axis (the interval gap of the corner projections) wins only
    # when it separates more by the margin 1e-4 (1 + |face separation|)
    cx, cy = _corners(*boxes[0]), _corners(*boxes[1])
    edge = None
    for i, j in itertools.product(range(3), range(3)):
        L = np.cross(boxes[0][1][:, i], boxes[1][1][:, j])
        if np.linalg.norm(L) < 1e-5:
            continue
        L /= np.linalg.norm(L)
        px, py = cx @ L, cy @ L
        gap = max(py.min() - px.max(), px.min() - py.max())
        edge = gap if edge is None else max(edge, gap)
    if edge is not None and edge > best[0] + 1e-4 * (1 + abs(best[0])):
        assert cnt == 1          # an edge contact (pinned by the edge test)
        return
    _, zr, k, nR = best
    cR, RR, hR = boxes[zr]
    cI, RI, hI = boxes[1 - zr]
    fc = cR + nR * hR[k]
    u, v = RR[:, (k + 1) % 3], RR[:, (k + 2) % 3]
    hu, hv = hR[(k + 1) % 3], hR[(k + 2) % 3]
    rect = [np.array(p) for p in ((hu, hv), (-hu, hv), (-hu, -hv), (hu, -hv))]
    # incident face: the other box's face whose outward normal is most anti-parallel to nR
    ki = int(np.argmax(np.abs(RI.T @ nR)))
    sgn = -np.sign(RI[:, ki] @ nR)
    fcI = cI + RI[:, ki] * (hI[ki] * sgn)
    k1, k2 = (ki + 1) % 3, (ki + 2) % 3
    V = [fcI + RI[:, k1] * (s1 * hI[k1]) + RI[:, k2] * (s2 * hI[k2]) for s1, s2 in ((1, 1), (-1, 1), (-1, -1), (1, -1))]
    inc = [np.array([(p - fc) @ u, (p - fc) @ v]) for p in V]
    nI = RI[:, ki] * sgn

    def height(xy2):
        """Height above the reference plane of the incident plane's point over (x, y)."""
        base = fc + u * xy2[0] + v * xy2[1]
        return ((fcI - base) @ nI) / (nR @ nI)
    cand = [(p, height(p)) for p in _overlap_polygon(inc, rect)]
    below = [(p, hgt) for p, hgt in cand if hgt < OFF]
    if not below:
        assert cnt == 0
        return
    got = []
    for i in range(cnt):
        a, b = d.contact_ids[0, i]
        g = d.contact_geom[0, i]
        assert (a, b) == (0, 1)
        pX = xb + Rb @ g[3:6]              # on the dynamic box
        pY = g[6:9]                        # on the static box (world)
        pR, pI = (pX, pY) if zr == 0 else (pY, pX)
        np.testing.assert_allclose(g[:3], nR if zr == 0 else -nR, atol=TOL_FRAME)
        got.append((np.array([(pR - fc) @ u, (pR - fc) @ v]), g[9]))
        assert abs((pI - pR) @ nR - g[9]) < TOL_FRAME
        assert abs((pR - fc) @ nR) < TOL_FRAME
    if len(below) <= 4:
        assert cnt == len(below)
        for p, hgt in below:
            assert min(np.linalg.norm(p - q) + abs(hgt - s) for q, s in got) < TOL_FRAME
        return
    assert cnt == 4
    # every chosen point is a candidate
    for q, s in got:
        assert min(np.linalg.norm(p - q) + abs(hgt - s) for p, hgt in below) < TOL_FRAME
    P = np.array([p for p, _ in below])
    Hh = np.array([hgt for _, hgt in below])
    (q0, s0), (q1, _), (q2, _), (q3, _) = got
    assert abs(s0 - Hh.min()) < TOL_FRAME                                        # deepest
    assert abs(np.linalg.norm(q1 - q0) - np.linalg.norm(P - q0, axis=1).max()) < TOL_FRAME   # farthest from it
    ex = q1 - q0
    area = ex[0] * (P[:, 1] - q0[1]) - ex[1] * (P[:, 0] - q0[0])
    a2 = ex[0] * (q2[1] - q0[1]) - ex[1] * (q2[0] - q0[0])
    assert abs(abs(a2) - np.abs(area).max()) < TOL_FRAME                        # largest triangle
    a3 = ex[0] * (q3[1] - q0[1]) - ex[1] * (q3[0] - q0[0])
    assert a3 * a2 <= TOL_FRAME                                             # on the other side
    assert abs(-np.sign(a2) * a3 - (-np.sign(a2) * area).max()) < TOL_FRAME      # farthest there


def _edges(c, R, h):
    out = []
    for ax in range(3):
        o1, o2 = [k for k in range(3) if k != ax]
        for s1, s2 in itertools.product((-1, 1), repeat=2):
            m = c + R[:, o1] * (s1 * h[o1]) + R[:, o2] * (s2 * h[o2])
            out.append((m, R[:, ax], h[ax]))
    return out


@pytest.mark.parametrize("seed", range(8))
def test_box_box_edge_contact_is_the_closest_edge_pair(seed):
    rng = np.random.default_rng(300 + seed)
    h = rng.uniform(0.04, 0.08)
    jitter = rng.uniform(-0.05, 0.05, 2)
    qA = axis_angle((1, 0, 0), np.pi / 4 + jitter[0])
    qB = axis_angle((0, 1, 0), np.pi / 4 + jitter[1])
    RA, RB = _rot(qA), _rot(qB)
    topA = np.max((RA @ (np.array(list(itertools.product((-1, 1), repeat=3))) * h).T)[2])
    lowB = np.min((RB @ (np.array(list(itertools.product((-1, 1), repeat=3))) * h).T)[2])
    shift = rng.uniform(-0.3, 0.3, 2) * h
    zb = 0.5 + topA - lowB - rng.uniform(0.0005, 0.003)
    e = env()
    e.body(S.BOX, (h, h, h), 1.0, (0.0, 0.0, 0.5), qA)
    e.body(S.BOX, (h, h, h), 1.0, (shift[0], shift[1], zb), qB)
    sc = scene_from_envs([e])
    d = _detect(sc)
    assert d.contact_count[0] == 1
    g = d.contact_geom[0, 0]
    xa, Ra = _pose(sc, 0)
    xb, Rb = _pose(sc, 1)
    ha, hb = sc.body_dims[0, :3].astype(np.float64), sc.body_dims[1, :3].astype(np.float64)
    pa, pb = xa + Ra @ g[3:6], xb + Rb @ g[6:9]
    best = None
    for (ca, da, la), (cb, db, lb) in itertools.product(_edges(xa, Ra, ha), _edges(xb, Rb, hb)):
        if np.linalg.norm(np.cross(da, db)) < 1e-3:
            continue
        p, q, _, _ = _seg_seg(ca, da, la, cb, db, lb)
        dd = np.linalg.norm(q - p)
        if best is None or dd < best[0]:
            best = (dd, p, q)
    _, p, q = best
    np.testing.assert_allclose(pa, p, atol=1e-6)
    np.testing.assert_allclose(pb, q, atol=1e-6)
    assert abs(g[9] - g[:3] @ (pb - pa)) < TOL_FRAME
    assert abs(abs(g[9]) - np.linalg.norm(q - p)) < 1e-6
    assert g[9] < 0


@pytest.mark.parametrize("seed", range(8))
def test_sphere_centre_inside_a_box_is_pushed_out_of_the_nearest_face(seed):
    """A sphere whose centre lies inside a box: one contact, normal along the
    nearest face's outward normal (towards the box), separation minus the
    distance to that face minus the radius (brute force over the six faces)."""
    rng = np.random.default_rng(400 + seed)
    h = rng.uniform(0.05, 0.2, 3)
    q = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    loc = rng.uniform(-0.8, 0.8, 3) * h
    R = _rot(q)
    c = np.array([0.0, 0.0, 1.0])
    r = rng.uniform(0.01, 0.04)
    e = env()
    e.body(S.SPHERE, (r,), 0.5, tuple(c + R @ loc))
    e.static(tuple(c), tuple(h), q)
    sc = scene_from_envs([e])
    d = _detect(sc)
    assert d.contact_count[0] == 1
    g = d.contact_geom[0, 0]
    pst = sc.static_pose[0].astype(np.float64)
    xb, Rb, hb = pst[:3], _rot(pst[3:]), sc.static_half[0].astype(np.float64)
    xs = sc.pos[0].astype(np.float64)
    rad = float(sc.body_dims[0, 0])
    faces = []
    for k in range(3):
        for sg in (-1.0, 1.0):
            nk = Rb[:, k] * sg
            faces.append((float((xb + nk * hb[k] - xs) @ nk), nk))
    dist, nk = min(faces, key=lambda f: f[0])
    assert abs(g[9] - (-dist - rad)) < TOL_FRAME
    np.testing.assert_allclose(g[:3], -nk, atol=TOL_FRAME)     # from the sphere into the box
    np.testing.assert_allclose(g[6:9], xs + nk * dist, atol=TOL_FRAME)   # the face point (world)


@pytest.mark.parametrize("seed", range(10))
def test_capsule_entering_a_box_contacts_at_its_ends_and_entry(seed):
    """A capsule whose segment enters a box: the manifold holds the sphere-box
    contacts of both end caps and of the sphere at the first point where the
    segment meets the box (the first minimiser of the segment's outside
    distance; dropped within 1 mm of an end), each with its signed distance
    (negative inside, from the nearest face) minus the radius."""
    rng = np.random.default_rng(500 + seed)
    h = rng.uniform(0.05, 0.15, 3)
    qb = axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
    Rb = _rot(qb)
    cb = np.array([0.0, 0.0, 1.0])
    r, L = rng.uniform(0.02, 0.04), rng.uniform(0.06, 0.12)
    # the segment crosses a face near its middle, one end inside, one outside
    k = int(rng.integers(3))
    sg = rng.choice([-1.0, 1.0])
    loc = rng.uniform(-0.5, 0.5, 3) * h
    loc[k] = sg * h[k]
    dl = rng.normal(size=3) * 0.4
    dl[k] = sg if seed % 2 else -sg      # odd seeds start inside, even ones enter from outside
    ac = Rb @ (dl / np.linalg.norm(dl))
    cc = cb + Rb @ loc + ac * rng.uniform(-0.3, 0.3) * L
    e = env()
    e.body(S.CAPSULE, (r, L), 0.5, tuple(cc), _quat_from_x(ac))
    e.static(tuple(cb), tuple(h), qb)
    sc = scene_from_envs([e])
    d = _detect(sc)
    xc, Rc = _pose(sc, 0)
    rad, Lc = float(sc.body_dims[0, 0]), float(sc.body_dims[0, 1])
    pst = sc.static_pose[0].astype(np.float64)
    xb, Rbs, hb = pst[:3], _rot(pst[3:]), sc.static_half[0].astype(np.float64)
    a = Rc[:, 0]

    def outside(t):
        l = Rbs.T @ (xc + a * t - xb)
        return float(np.linalg.norm(l - np.clip(l, -hb, hb)))
    ts = np.linspace(-Lc, Lc, 40001)
    ov = np.array([outside(t) for t in ts])
    assert (ov == 0).any() and (ov[0] > 0 or ov[-1] > 0)
    i = int(np.argmax(ov == 0))
    if i == 0:
        t_entry = -Lc
    else:
        lo, hi = ts[i - 1], ts[i]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if outside(mid) > 0:
                lo = mid
            else:
                hi = mid
        t_entry = hi
    want = [-Lc, Lc] + ([t_entry] if (t_entry + Lc) > 1e-3 + 1e-6 and (Lc - t_entry) > 1e-3 + 1e-6 else [])
    want = [t for t in want if _point_box(xc + a * t, xb, Rbs, hb)[0] - rad < OFF]
    cnt = d.contact_count[0]
    assert cnt == len(want)
    got = []
    for j in range(cnt):
        g = d.contact_geom[0, j]
        centre = xc + Rc @ g[3:6] - g[:3] * rad
        t = float(a @ (centre - xc))
        got.append(t)
        assert abs(g[9] - (_point_box(centre, xb, Rbs, hb)[0] - rad)) < TOL_FRAME
    for t in want:
        assert min(abs(t - u) for u in got) < 1e-6


def test_box_box_clipping_never_reaches_its_vertex_cap_on_near_degenerate_faces():
    """The incident face (a quad) is clipped by the reference face's four side
    planes one at a time; a convex polygon gains at most one vertex per
    half-plane, so the result has at most 4 + 4 = 8 vertices in exact
    arithmetic, the clipper's cap. Rounding could in principle add sign
    changes where vertices lie within rounding of a side plane; these
    near-degenerate cases (equal or nearly equal faces, edges aligned to
    within rounding, tilts of 1e-7 to 1e-4 rad, incident faces larger than
    the reference face) are run in FP32 and FP64 and the cap must drop
    nothing."""
    rng = np.random.default_rng(77)
    envs = []
    for k in range(600):
        h = rng.uniform(0.03, 0.2, 3)
        e = env()
        e.static((0.0, 0.0, 0.5), tuple(h), axis_angle((0, 0, 1), float(rng.choice([0.0, np.pi / 2, rng.uniform(0, np.pi)]))))
        mode = k % 3
        if mode == 0:      # same footprint, aligned edges
            hb = h.copy()
        elif mode == 1:    # edges off by about rounding
            hb = h * (1.0 + rng.choice([-1.0, 1.0], 3) * rng.uniform(0, 1e-6, 3))
        else:              # incident face larger than the reference face
            hb = h * np.array([1.5, 1.3, 1.0])
        tilt = axis_angle(rng.normal(size=3), float(10.0 ** rng.uniform(-7, -4)))
        w0, x0, y0, z0 = tilt
        w1, x1, y1, z1 = e.statics[0][0][3:]
        q = (w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1, w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
             w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1, w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1)
        shift = rng.choice([0.0, 1.0], 2) * rng.uniform(-1e-6, 1e-6, 2)
        R = _rot(e.statics[0][0][3:])
        c = np.array([0.0, 0.0, 0.5]) + R @ np.array([shift[0], shift[1], h[2] + hb[2] - 0.002])
        e.body(S.BOX, tuple(hb), 1.0, tuple(c), quat=q)
        envs.append(e)
    sc = scene_from_envs(envs)
    c = cfg(max_contacts=8, max_pairs=4)
    before = oracle.clip_cap_drops()
    for prec in ("f32", "f64"):
        d = oracle.detect(sc, c, sc.pos, sc.quat, prec)
        assert (d.contact_count >= 1).all()
    assert oracle.clip_cap_drops() == before
