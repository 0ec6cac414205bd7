"""Seeded synthetic per-step records for the event labeling (Sec. 3.3).

Stands in for the paper's policy rollouts (its HAB episodes and trained
policies are not in this container). Each trajectory acts out a randomly
drawn script of the subtask -- reaching, touching, grasping and dropping,
carrying towards a goal, releasing, pulling an articulation, collisions
building up, success switching on and off -- so that every success and
failure mode occurs. Records are float32 arrays [T, N] in step-major order
(the layout the labeling kernel reads), flags uint8 [T, N] (bit 0 grasped,
bit 1 success), per-trajectory lengths, articulation ranges and fridge flags.
Holds none of the labeling arithmetic.
"""
from __future__ import annotations

import numpy as np

PICK, PLACE, OPEN, CLOSE = 0, 1, 2, 3


def _toggles(rng, T, n_on, start):
    """A 0/1 series that switches on at `start` and toggles at n_on random later times."""
    x = np.zeros(T, np.uint8)
    if start >= T:
        return x
    times = np.sort(rng.integers(start + 1, T + 1, size=n_on)) if n_on else np.zeros(0, np.int64)
    state, t0 = 1, start
    for t in list(times) + [T]:
        x[t0:t] = state
        state ^= 1
        t0 = t
    return x


def make(task: int, num: int, steps: int, seed: int = 0, min_len: float = 0.6) -> dict:
    rng = np.random.default_rng(np.random.PCG64(90001 + 17 * task + 1000003 * seed))
    T, N = steps, num
    force = np.zeros((T, N), np.float32)
    cumcol = np.zeros((T, N), np.float32)
    dist = np.zeros((T, N), np.float32)
    artq = np.zeros((T, N), np.float32)
    flags = np.zeros((T, N), np.uint8)
    length = rng.integers(int(min_len * T), T + 1, size=N).astype(np.int32)
    art_range = np.zeros((N, 2), np.float32)
    fridge = rng.integers(0, 2, size=N).astype(np.uint8)
    limit = {PICK: 5000.0, PLACE: 7500.0, OPEN: 10000.0, CLOSE: 10000.0}[task]
    for k in range(N):
        # collisions: per-step increments with a trajectory-specific scale
        scale = limit / T * np.exp(rng.uniform(np.log(0.05), np.log(4.0)))
        inc = rng.exponential(scale, size=T) * (rng.random(T) < 0.5)
        inc[0] = 0.0
        cumcol[:, k] = np.cumsum(inc)
        # force: zero until first contact, then on/off periods
        t_contact = rng.integers(1, T + T // 3)
        on = _toggles(rng, T, int(rng.integers(0, 2)), t_contact)
        force[:, k] = on * rng.uniform(0.5, 40.0, size=T)
        g = np.zeros(T, np.uint8)
        if task in (PICK, PLACE):
            if task == PLACE and rng.random() < 0.85:
                g = _toggles(rng, T, int(rng.integers(0, 4)), 0)          # starts holding x
            else:
                g = _toggles(rng, T, int(rng.integers(0, 4)), int(t_contact + rng.integers(0, 10)))
        s = _toggles(rng, T, int(rng.integers(0, 3)), int(rng.integers(T // 4, T + T // 2)))
        if task == PLACE:
            d0 = rng.uniform(0.02, 0.8)
            d1 = rng.uniform(0.0, 0.4)
            path = np.linspace(d0, d1, T) + np.cumsum(rng.normal(0.0, 0.02, size=T))
            dist[:, k] = np.abs(path)
        if task in (OPEN, CLOSE):
            qmax = rng.uniform(0.3, 1.6)
            art_range[k] = (0.0, qmax)
            q0 = 0.0 if task == OPEN else qmax * rng.uniform(0.7, 1.0)
            q1 = qmax * rng.uniform(0.0, 1.0) if task == OPEN else qmax * rng.uniform(-0.05, 0.6)
            path = np.linspace(q0, q1, T) + np.cumsum(rng.normal(0.0, 0.01 * qmax, size=T))
            artq[:, k] = np.clip(path, 0.0, qmax)
            artq[0, k] = q0
        # success holds only where the subtask's success condition can (Appendix A.4):
        # holding x (Pick), x released within 15 cm (Place), open / closed (Open / Close)
        if task == PICK:
            s &= g
        elif task == PLACE:
            s &= (1 - g) & (dist[:, k] <= 0.15).astype(np.uint8)
        elif task == OPEN:
            s &= (artq[:, k] >= (0.75 if fridge[k] else 0.9) * art_range[k, 1]).astype(np.uint8)
        else:
            s &= (artq[:, k] <= 0.01 * art_range[k, 1]).astype(np.uint8)
        flags[:, k] = g | (s << 1)
    traj = dict(cumcol=cumcol, flags=flags, length=length)
    if task in (PICK, OPEN, CLOSE):
        traj["force"] = force
    if task == PLACE:
        traj["dist"] = dist
    if task in (OPEN, CLOSE):
        traj["artq"] = artq
        traj["art_range"] = art_range
        traj["art_fridge"] = fridge
    return traj
