"""Differentiable rollouts of the batched step (torch.autograd.Function).

`rollout(sim, state, targets, mass, checkpoint_every)` steps the batch
through targets[0..T) and returns the final state. Its backward pass keeps
only every k-th state from the forward pass (step checkpointing): for each
segment, last first, it restores the segment's start state, re-runs the
segment with the library recording a tape, and reverses the recorded steps
with msh_backward. The forward pass records the last segment itself and
pauses the tape, so the backward pass reverses that segment without a
re-run when nothing has touched the tape in between. Memory is O(T/k
states + k tapes).

`mass` must hold the scene's body masses (the library derived the inverse
masses and inertias from them at msh_create); only its gradient is used.
"""
from __future__ import annotations

import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, targets, k, pos, quat, linvel, angvel, mass):
        T = int(targets.shape[0])
        k = max(1, min(int(k), T))
        sim.set_tape(0)
        for dst, src in ((sim.pos, pos), (sim.quat, quat), (sim.linvel, linvel), (sim.angvel, angvel)):
            dst.copy_(src)
        ckpts = []
        last = ((T - 1) // k) * k          # first step of the last segment
        for t in range(T):
            if t % k == 0:
                ckpts.append(tuple(x.clone() for x in (sim.pos, sim.quat, sim.linvel, sim.angvel)))
            if t == last:
                sim.set_tape(k)             # record the last segment now
            sim.step(targets[t])
        sim.tape_record(False)              # keep it, record nothing else
        ctx.token = object()
        sim.tape_owner = ctx.token
        ctx.sim, ctx.k, ctx.T, ctx.ckpts, ctx.recorded = sim, k, T, ckpts, T - last
        ctx.save_for_backward(targets)
        return tuple(x.clone() for x in (sim.pos, sim.quat, sim.linvel, sim.angvel))

    @staticmethod
    def backward(ctx, gpos, gquat, glv, gav):
        (targets,) = ctx.saved_tensors
        sim, k, T = ctx.sim, ctx.k, ctx.T
        like = (sim.pos, sim.quat, sim.linvel, sim.angvel)
        adj = tuple((g if g is not None else torch.zeros_like(x)).contiguous().float()
                    for g, x in zip((gpos, gquat, glv, gav), like))
        adj_targets = torch.zeros_like(targets)
        adj_mass = torch.zeros(sim.scene.num_bodies, dtype=torch.float32, device=sim.device)
        nseg = (T + k - 1) // k
        kept = sim.tape_owner is ctx.token and sim.tape_count == ctx.recorded
        for seg in reversed(range(nseg)):
            t0, t1 = seg * k, min(T, seg * k + k)
            if not (kept and seg == nseg - 1):
                for dst, src in zip((sim.pos, sim.quat, sim.linvel, sim.angvel), ctx.ckpts[seg]):
                    dst.copy_(src)
                sim.set_tape(k)
                for t in range(t0, t1):
                    sim.step(targets[t])
            for t in reversed(range(t0, t1)):
                adj = sim.backward(adj, adj_targets[t], adj_mass)
        sim.set_tape(0)        # stop recording; the tape memory is kept for the next backward pass
        return (None, adj_targets, None) + adj + (adj_mass,)


def rollout(sim, state, targets, mass, checkpoint_every: int = 8):
    """Final (pos, quat, linvel, angvel) after len(targets) steps, differentiable
    w.r.t. the initial state, the targets [T, E, max_dof] and `mass` [B]."""
    pos, quat, linvel, angvel = state
    return _Rollout.apply(sim, targets, checkpoint_every, pos, quat, linvel, angvel, mass)


def goal_loss(sim, pos):
    """Per-env squared distance of each env's goal body to its goal position."""
    sc = sim.scene
    idx = torch.as_tensor(sc.body_off[:-1] + sc.goal_body, device=pos.device, dtype=torch.long)
    goal = torch.as_tensor(sc.goal_pos, device=pos.device, dtype=torch.float32)
    d = pos[idx] - goal
    return (d * d).sum(dim=1)
