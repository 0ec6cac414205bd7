"""Element-wise comparison of one-step adjoints on the pieces of a piecewise
smooth step.

The step takes branch decisions (impulse clamps, joint-limit and contact-bias
cases); its adjoint is the derivative of the piece its own primal values
select. A decision taken within rounding of its threshold -- a friction row
that has converged onto its cone, a normal impulse that has converged to
zero -- is fragile: another correct FP32 evaluation may take it the other
way, and both one-sided derivatives are correct. The oracle reports its
fragile decisions (margins below a rounding-level threshold) and can take
any set of them the other way.

`check_env` compares a GPU adjoint of one env with the oracle's on the
oracle's own piece; when they differ it searches for a set of fragile
decisions to re-decide (single decisions, or all fragile decisions of one
solver row forced clamped or forced free) that makes them agree element by
element. Agreement on the oracle's own piece, or on a piece reached by
re-deciding only fragile decisions, is a pass; anything else fails.
"""
import numpy as np

import oracle

KINDS = ("pos", "quat", "linvel", "angvel", "targets", "mass")
RTOL, ATOL, FLOOR = 2e-3, 2e-3, 1e-5
# decision margins (relative to the update's magnitude) taken as rounding
# level; the search runs with the tighter one first
FRAGILE = (1e-5, 1e-4)
MAX_ROUNDS = 12


def tangential(g, q):
    """The part of a quaternion adjoint tangent to the unit sphere at q."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    g = np.asarray(g, np.float64)
    return g - (g * q).sum(1, keepdims=True) * q


def env_ratio(ref, got, quat):
    """Worst ratio of |got - ref| to the tolerance over one env's elements:
    RTOL of the element, ATOL of the largest of its kind in the env, FLOOR
    of the env's largest element of any kind."""
    r = {k: np.asarray(ref[k], np.float64) for k in KINDS}
    g = {k: np.asarray(got[k], np.float64) for k in KINDS}
    r["quat"] = tangential(r["quat"], quat)
    g["quat"] = tangential(g["quat"], quat)
    envmax = max(float(np.abs(r[k]).max(initial=0.0)) for k in KINDS)
    worst, where = 0.0, None
    for k in KINDS:
        if r[k].size == 0:
            continue
        tol = RTOL * np.abs(r[k]) + ATOL * np.abs(r[k]).max() + FLOOR * envmax + 1e-30
        q = float((np.abs(g[k] - r[k]) / tol).max())
        if q > worst or not np.isfinite(q):
            worst, where = q, k
    return worst, where


def _env_dict(r, i):
    return {k: (getattr(r, k)[i] if k == "targets" else getattr(r, k)) for k in KINDS}


def check_env(sub, cfg, state, targets, seed, got):
    """sub: a one-env scene; state/targets/seed: that env's FP32 inputs and
    seed; got: the GPU's adjoints of that env (dict of KINDS). Returns
    (ratio, flips) with flips the re-decided fragile decisions (empty when
    the oracle's own piece agrees); ratio <= 1 means agreement."""
    best = None
    for delta in FRAGILE:
        cur, flips = _search(sub, cfg, state, targets, seed, got, delta)
        if best is None or cur < best[0]:
            best = (cur, flips)
        if cur <= 1.0:
            break
    return best


def _search(sub, cfg, state, targets, seed, got, delta):
    """Greedy search over the fragile decisions of margin below delta."""
    quat = np.asarray(state[1], np.float64)
    base = oracle.step_vjp(sub, cfg, state, targets, seed, "f32", fragile=True, delta=delta, kmax=4096)
    cur, _ = env_ratio(_env_dict(base, 0), got, quat)
    if cur <= 1.0:
        return cur, []
    idx, site, choice = base.fragile[0], base.fragile_site[0], base.fragile_choice[0]
    cands = [[int(i)] for i in idx]
    for s in sorted(set(int(x) for x in site if x >= 0)):
        to_clamped = [int(i) for i, x, c in zip(idx, site, choice) if x == s and c == 0]
        to_free = [int(i) for i, x, c in zip(idx, site, choice) if x == s and c == 1]
        for grp in (to_clamped, to_free):
            if len(grp) > 1:
                cands.append(grp)
    flips = []
    for _ in range(MAX_ROUNDS):
        best = None
        for c in cands:
            trial = sorted(set(flips) | set(c))
            if trial == flips:
                continue
            r = oracle.step_vjp(sub, cfg, state, targets, seed, "f32", flips=[trial])
            q, _ = env_ratio(_env_dict(r, 0), got, quat)
            if best is None or q < best[0]:
                best = (q, trial)
        if best is None or best[0] >= cur:
            break
        cur, flips = best
        if cur <= 1.0:
            break
    return cur, flips
