"""Oracle of the automated event labeling and trajectory categorization
(paper Sec. 3.3 and Appendix A.5) -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU legs use this module. It
restates the appendix's definitions with plain Python lists, one trajectory at
a time: for t = 1..n, every event of the subtask is evaluated in the listed
order from the records at t-1 and t and appended when true; the mode is then
read off the chronological event list with the appendix's boolean formulas.

Per-step records of one trajectory (t = 0 is the initial state):
  force[t]   |F_{ee,x,t}|, the end-effector/target pairwise force in N
  cumcol[t]  the robot's cumulative collision force in N
  dist[t]    distance of the target to its goal in m (Place)
  artq[t]    the articulation's joint position (Open, Close)
  grasped[t], success[t]  booleans

Readings where the text is ambiguous or garbled (each also in the design notes):
  L1 e_contact's second clause reads |F_t| >= 0, which always holds; Sec. 3.3
     defines Contact as a nonzero pairwise force, so it is |F_t| > 0.
  L2 i_{subtask,event} is the index of the event in E; for an event that occurs
     more than once it is its LAST occurrence (Sec. 3.3 uses "maximal i, j").
  L3 d^a_b is printed as a squared norm "in m"; the 15 cm goal radius is a
     distance, so d is the Euclidean distance (the caller's dist).
  L4 Pick winding success "(contact, grasped, ..., success)": the list starts
     with contact, grasped and ends with success.
  L5 Open/Close success mode iii prints "excessive_collisions not in E"; the
     mode's text ("exceeds collision threshold afterwards") means "in E".
  L6 Close's slightly_closed prints q_qmin for a_qmin.
  L7 modes are tested in the listed order and the first that holds is the
     label; 0 means none holds (the appendix calls the modes exhaustive).
  L8 thresholds are formed and compared in FP32 (the precision of the
     records and of the kernel), e.g. 0.9 (qmax - qmin) + qmin as an FP32
     multiply then add.
"""
from __future__ import annotations

import numpy as np

PICK, PLACE, OPEN, CLOSE = 0, 1, 2, 3
f32 = np.float32

# event names per subtask, in the appendix's evaluation order
EVENTS = {
    PICK: ["contact", "grasped", "dropped", "success", "excessive_collisions"],
    PLACE: ["grasped", "obj_at_goal", "released_at_goal", "released_outside_goal", "obj_left_goal", "success",
            "excessive_collisions"],
    OPEN: ["contact", "opened", "slightly_opened", "closed", "success", "excessive_collisions"],
    CLOSE: ["contact", "closed", "slightly_closed", "opened", "success", "excessive_collisions"],
}
# default collision thresholds (Appendix A.4: Pick 5000 N, Place 7500 N, Open/Close 10000 N)
COLLISION_LIMIT = {PICK: 5000.0, PLACE: 7500.0, OPEN: 10000.0, CLOSE: 10000.0}
GOAL_RADIUS = 0.15


def _frac(frac, qmin, qmax):
    """frac (qmax - qmin) + qmin in FP32 (L8)."""
    return float(f32(f32(frac) * f32(f32(qmax) - f32(qmin))) + f32(qmin))


def _open(q, qmin, qmax, fridge):
    """1_open(a): a_q >= a_ofrac (a_qmax - a_qmin) + a_qmin, a_ofrac 0.75 for a fridge else 0.9 (A.4)."""
    return q >= _frac(0.75 if fridge else 0.9, qmin, qmax)


def _closed(q, qmin, qmax):
    """1_close(a): a_q <= 0.01 (a_qmax - a_qmin) + a_qmin (A.4)."""
    return q <= _frac(0.01, qmin, qmax)


def events(task, rec, n, limit=None, goal_radius=GOAL_RADIUS, qmin=0.0, qmax=1.0, fridge=False):
    """Chronological event list (names) of one trajectory over t = 1..n-1.

    rec: dict of per-step lists force, cumcol, dist, artq, grasped, success."""
    lim = float(f32(COLLISION_LIMIT[task] if limit is None else limit))
    goal_radius = float(f32(goal_radius))
    F, C, d, q = rec.get("force"), rec["cumcol"], rec.get("dist"), rec.get("artq")
    g, s = rec.get("grasped"), rec["success"]
    E = []
    for t in range(1, n):
        ev = {}
        exc = C[t - 1] <= lim and C[t] > lim
        if task == PICK:
            ev["contact"] = F[t - 1] == 0 and F[t] > 0                                   # L1
            ev["grasped"] = (not g[t - 1]) and g[t]
            ev["dropped"] = g[t - 1] and not g[t]
        elif task == PLACE:
            ev["grasped"] = (not g[t - 1]) and g[t]
            ev["obj_at_goal"] = d[t - 1] > goal_radius and d[t] <= goal_radius
            ev["released_at_goal"] = d[t] <= goal_radius and g[t - 1] and not g[t]
            ev["released_outside_goal"] = d[t] > goal_radius and g[t - 1] and not g[t]
            ev["obj_left_goal"] = d[t - 1] <= goal_radius and d[t] > goal_radius
        elif task == OPEN:
            o0, o1 = _open(q[t - 1], qmin, qmax, fridge), _open(q[t], qmin, qmax, fridge)
            so0 = q[t - 1] >= _frac(0.1, qmin, qmax)
            so1 = q[t] >= _frac(0.1, qmin, qmax)
            ev["contact"] = F[t - 1] == 0 and F[t] > 0                                   # L1
            ev["opened"] = (not o0) and o1
            ev["slightly_opened"] = (not so0) and so1
            ev["closed"] = o0 and not o1
        else:
            c0, c1 = _closed(q[t - 1], qmin, qmax), _closed(q[t], qmin, qmax)
            thr = float(f32(q[0]) - f32(f32(0.05) * f32(f32(qmax) - f32(qmin))))       # L6
            sc0, sc1 = q[t - 1] < thr, q[t] < thr
            ev["contact"] = F[t - 1] == 0 and F[t] > 0                                   # L1
            ev["closed"] = (not c0) and c1
            ev["slightly_closed"] = (not sc0) and sc1
            ev["opened"] = c0 and not c1
        ev["success"] = (not s[t - 1]) and s[t]
        ev["excessive_collisions"] = exc
        for name in EVENTS[task]:
            if ev[name]:
                E.append(name)
    return E


def idx(E, name):
    """i_{subtask,event}: index of the event in E (its last occurrence, L2), -1 if absent."""
    last = -1
    for i, e in enumerate(E):
        if e == name:
            last = i
    return last


def label(task, E, d0=None, goal_radius=GOAL_RADIUS):
    """The success or failure mode (1-based roman numeral of Appendix A.5), 0 if none (L7)."""
    goal_radius = float(f32(goal_radius))
    exc = "excessive_collisions" in E
    i = lambda name: idx(E, name)   # noqa: E731
    if task == PICK:
        if "success" in E:
            if E == ["contact", "grasped", "success"]:
                return 1                                                                  # straightforward
            if len(E) > 3 and E[:2] == ["contact", "grasped"] and E[-1] == "success" and not exc:   # L4
                return 2                                                                  # winding
            if "dropped" in E and i("dropped") > i("grasped") and not exc:
                return 3                                                                  # success then drop
            if exc:
                return 4                                                                  # success then excessive
            return 0
        if exc:
            return 5
        if E == []:
            return 6                                                                      # mobility
        if E == ["contact"]:
            return 7                                                                      # can't grasp
        if "dropped" in E and i("dropped") > i("grasped") and not exc:
            return 8                                                                      # drop failure
        if "grasped" in E and i("grasped") > i("dropped") and not exc:
            return 9                                                                      # too slow
        return 0
    if task == PLACE:
        near0 = d0 <= goal_radius
        if "success" in E:
            if (len(E) <= 4 and ("released_at_goal" in E or near0) and i("obj_left_goal") <= i("obj_at_goal")
                    and not exc):
                return 1                                                                  # place in goal
            if (len(E) <= 4 and ("released_outside_goal" in E or not near0)
                    and i("obj_left_goal") <= i("obj_at_goal") and not exc):
                return 2                                                                  # dropped to goal
            if i("obj_at_goal") < i("obj_left_goal") and not exc:
                return 3                                                                  # dubious
            if len(E) > 4 and i("obj_at_goal") > i("obj_left_goal") and not exc:
                return 4                                                                  # winding
            if exc:
                return 5                                                                  # success then excessive
            return 0
        if exc:
            return 6
        if E == []:
            return 7                                                                      # didn't grasp
        if len(E) > 0 and "obj_at_goal" not in E:
            return 8                                                                      # didn't reach goal
        placed_latest = (len(E) <= 2 and near0) or (
            i("released_at_goal") > i("released_outside_goal") and i("released_at_goal") > i("grasped"))
        if "obj_at_goal" in E and placed_latest and i("obj_left_goal") > i("obj_at_goal"):
            return 9                                                                      # place in goal failure
        dropped_latest = (len(E) <= 2 and not near0) or (
            i("released_outside_goal") > i("released_at_goal") and i("released_outside_goal") > i("grasped"))
        if "obj_at_goal" in E and dropped_latest and i("obj_left_goal") > i("obj_at_goal"):
            return 10                                                                     # dropped to goal failure
        if ("obj_at_goal" in E and i("grasped") > i("released_at_goal")
                and i("grasped") > i("released_outside_goal")):
            return 11                                                                     # won't let go
        return 12                                                                         # too slow
    if task == OPEN:
        if "success" in E:
            if not exc and i("opened") > i("closed"):
                return 1                                                                  # open success
            if not exc and i("opened") < i("closed"):
                return 2                                                                  # dubious
            if exc:                                                                       # L5
                return 3
            return 0
        if exc:
            return 4
        if "contact" not in E:
            return 5                                                                      # can't reach
        if "closed" in E and i("closed") > i("opened") and i("closed") > i("slightly_opened"):
            return 6                                                                      # closed after open
        if i("slightly_opened") > i("opened") and i("slightly_opened") > i("closed"):
            return 7                                                                      # slightly opened
        if "opened" in E:
            return 8                                                                      # too slow
        return 9                                                                          # can't open
    if "success" in E:
        if not exc and i("closed") > i("opened"):
            return 1                                                                      # close success
        if not exc and i("closed") < i("opened"):
            return 2                                                                      # dubious
        if exc:                                                                           # L5
            return 3
        return 0
    if exc:
        return 4
    if "contact" not in E:
        return 5                                                                          # can't reach
    if "closed" in E and i("opened") > i("closed") and i("opened") > i("slightly_closed"):
        return 6                                                                          # opened after closed
    if i("slightly_closed") > i("closed") and i("slightly_closed") > i("opened"):
        return 7                                                                          # slightly closed
    if "closed" in E:
        return 8                                                                          # too slow
    return 9                                                                              # can't close


def label_batch(task, traj, limit=None, goal_radius=GOAL_RADIUS):
    """Events and labels of every trajectory of a batch.

    traj: dict of numpy arrays force/cumcol/dist/artq [T, N] (float), flags
    [T, N] (bit 0 grasped, bit 1 success), optional length [N], art_range [N, 2],
    art_fridge [N]. Returns (event lists, labels)."""
    T, N = traj["cumcol"].shape
    out_e, out_l = [], []
    for k in range(N):
        n = int(traj["length"][k]) if traj.get("length") is not None else T
        fl = traj["flags"][:, k]
        rec = {"cumcol": [float(x) for x in traj["cumcol"][:, k]],
               "grasped": [bool(x & 1) for x in fl], "success": [bool(x & 2) for x in fl]}
        for key in ("force", "dist", "artq"):
            if traj.get(key) is not None:
                rec[key] = [float(x) for x in traj[key][:, k]]
        kw = {}
        if task in (OPEN, CLOSE):
            kw = dict(qmin=float(traj["art_range"][k, 0]), qmax=float(traj["art_range"][k, 1]),
                      fridge=bool(traj["art_fridge"][k]))
        E = events(task, rec, n, limit, goal_radius, **kw)
        d0 = rec["dist"][0] if task == PLACE else None
        out_e.append(E)
        out_l.append(label(task, E, d0, goal_radius))
    return out_e, out_l
