"""Scenario sharding across ranks (weak scaling) and the one exchange step.

Scenarios are independent, so rank r of N evaluates scenarios
[r*S, (r+1)*S) of one N*S-scenario set with no data-path communication; the
only exchange is the global FP64 mean, an all-reduce of (sum, count) pairs.
"""
from __future__ import annotations

import torch


def scenario_range(rank: int, world: int, per_rank: int) -> tuple[int, int]:
    """[s0, s1) of the global scenario set owned by `rank`."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return rank * per_rank, (rank + 1) * per_rank


def combine_mean(local_sum: float, local_count: int, group=None, device=None) -> float:
    """Global mean from per-rank FP64 sums (sum of sums / sum of counts)."""
    import torch.distributed as dist
    t = torch.tensor([float(local_sum), float(local_count)], dtype=torch.float64,
                     device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t[0] / t[1]) if t[1] > 0 else 0.0


def max_over_ranks(x: float, group=None, device=None) -> float:
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t[0])
