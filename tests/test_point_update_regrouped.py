"""The fused kernel updates a contact point's three rows (normal, then the
two friction rows, sequential impulses as reading C8 orders them) in a
regrouped form: the relative velocity at the point is formed once, each
later row's velocity component is moved by the earlier rows' impulse changes
through the couplings K(x, y) = J_x M^-1 J_y^T, and the point's total impulse
is applied to both bodies once. This pins that regrouping against the
row-by-row update in FP64 on random points: the same lambdas and body
velocities to rounding, with the clamps (normal at zero, friction at
+-mu*lambda_n) active and inactive."""
import numpy as np
import pytest


def _sym(rng):
    a = rng.normal(size=(3, 3))
    return a @ a.T + 0.5 * np.eye(3)


def _onb(n):
    sg = 1.0 if n[2] >= 0 else -1.0
    a = -1.0 / (sg + n[2])
    b = n[0] * n[1] * a
    return (np.array([1.0 + sg * n[0] * n[0] * a, sg * b, -sg * n[0]]),
            np.array([b, sg + n[1] * n[1] * a, -n[1]]))


def _setup(rng, dyn_b):
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    t1, t2 = _onb(n)
    d = [n, t1, t2]
    ra, rb = rng.normal(size=3) * 0.1, rng.normal(size=3) * 0.1
    ima, Ia = rng.uniform(0.5, 5.0), _sym(rng)
    imb, Ib = (rng.uniform(0.5, 5.0), _sym(rng)) if dyn_b else (0.0, np.zeros((3, 3)))

    def K(x, y):
        k = ima * x @ y + np.cross(ra, x) @ Ia @ np.cross(ra, y)
        if dyn_b:
            k += imb * x @ y + np.cross(rb, x) @ Ib @ np.cross(rb, y)
        return k

    m = [1.0 / K(x, x) for x in d]
    v = [rng.normal(size=3) for _ in range(4)]
    if not dyn_b:
        v[2] = np.zeros(3)
        v[3] = np.zeros(3)
    lam = np.array([rng.uniform(0.0, 0.2), rng.normal() * 0.05, rng.normal() * 0.05])
    bias = rng.normal() * 0.3
    return dict(d=d, ra=ra, rb=rb, ima=ima, Ia=Ia, imb=imb, Ib=Ib, K=K, m=m, v=v, lam=lam, bias=bias, dyn_b=dyn_b)


def _row_by_row(c, mu):
    va, wa, vb, wb = (x.copy() for x in c["v"])
    lam = c["lam"].copy()
    for r, d in enumerate(c["d"]):
        ca, cb = np.cross(c["ra"], d), np.cross(c["rb"], d)
        vn = d @ (vb - va) + cb @ wb - ca @ wa
        if r == 0:
            nl = max(lam[0] - c["m"][0] * (vn + c["bias"]), 0.0)
        else:
            lim = mu * lam[0]
            nl = min(max(lam[r] - c["m"][r] * vn, -lim), lim)
        dl = nl - lam[r]
        lam[r] = nl
        va = va - c["ima"] * dl * d
        wa = wa - dl * (c["Ia"] @ ca)
        if c["dyn_b"]:
            vb = vb + c["imb"] * dl * d
            wb = wb + dl * (c["Ib"] @ cb)
    return lam, (va, wa, vb, wb)


def _regrouped(c, mu):
    va, wa, vb, wb = c["v"]
    n, t1, t2 = c["d"]
    ra, rb, K = c["ra"], c["rb"], c["K"]
    vr = -(va + np.cross(wa, ra))
    if c["dyn_b"]:
        vr = vr + vb + np.cross(wb, rb)
    u0, u1, u2 = n @ vr, t1 @ vr, t2 @ vr
    l0, l1, l2 = c["lam"]
    nl0 = max(l0 - c["m"][0] * (u0 + c["bias"]), 0.0)
    d0 = nl0 - l0
    u1 += K(t1, n) * d0
    u2 += K(t2, n) * d0
    lim = mu * nl0
    nl1 = min(max(l1 - c["m"][1] * u1, -lim), lim)
    d1 = nl1 - l1
    u2 += K(t2, t1) * d1
    nl2 = min(max(l2 - c["m"][2] * u2, -lim), lim)
    d2 = nl2 - l2
    P = n * d0 + t1 * d1 + t2 * d2
    va2 = va - c["ima"] * P
    wa2 = wa - c["Ia"] @ np.cross(ra, P)
    vb2, wb2 = vb, wb
    if c["dyn_b"]:
        vb2 = vb + c["imb"] * P
        wb2 = wb + c["Ib"] @ np.cross(rb, P)
    return np.array([nl0, nl1, nl2]), (va2, wa2, vb2, wb2)


@pytest.mark.parametrize("dyn_b", [True, False])
@pytest.mark.parametrize("mu", [0.0, 0.5, 5.0])
def test_regrouped_point_update_equals_row_by_row(dyn_b, mu):
    rng = np.random.default_rng(7 + int(dyn_b) + int(10 * mu))
    clamps = set()
    for _ in range(400):
        c = _setup(rng, dyn_b)
        lam_r, v_r = _row_by_row(c, mu)
        lam_g, v_g = _regrouped(c, mu)
        scale = 1.0 + max(np.abs(x).max() for x in c["v"])
        assert np.allclose(lam_g, lam_r, rtol=0, atol=1e-12 * scale)
        for a, b in zip(v_g, v_r):
            assert np.allclose(a, b, rtol=0, atol=1e-11 * scale)
        lim = mu * lam_r[0]
        clamps.add((lam_r[0] == 0.0, abs(lam_r[1]) == lim, abs(lam_r[2]) == lim))
    assert len(clamps) >= 2   # both clamped and free rows were exercised
