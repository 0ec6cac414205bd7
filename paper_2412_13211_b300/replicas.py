"""Multi-GPU use of the batched step: replicas.

Environments are independent, so N GPUs run N replicas, each stepping its own
disjoint range of envs with no collective on the data path (weak scaling).
Only the benchmark's timing crosses ranks: the slowest rank's time bounds the
whole job.
"""
from __future__ import annotations


def env_range(envs_per_rank: int, rank: int) -> tuple[int, int]:
    """Global env indices [start, end) simulated by `rank`."""
    return rank * envs_per_rank, (rank + 1) * envs_per_rank


def slowest(seconds: float, device=None) -> float:
    """Max of `seconds` over all ranks of the default process group (the value
    itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(envs_per_rank: int, steps: int, seconds: float, world: int) -> float:
    """Env-steps per second of the whole job: all ranks' env-steps over the
    slowest rank's time."""
    return world * envs_per_rank * steps / seconds
