"""Host-side multi-GPU logic: independent problems shard across ranks, no
data-path collective.

A solve does not shard within itself without a transpose all-to-all, so the
multi-GPU path is replicas: each rank solves its own nests, the timed region is
bracketed by a barrier, and the job time is the slowest rank's.
"""
from __future__ import annotations

from typing import List, Sequence


def shard_by_cost(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the items rank `rank` owns: greedy longest-processing-time
    assignment of items (by cost) to the currently least-loaded rank; ties go
    to the lower rank.  Deterministic, so every rank computes the same split."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k))
    load = [0.0] * world
    owner = [0] * len(costs)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += float(costs[k])
    return [k for k in range(len(costs)) if owner[k] == rank]


def nest_cost(n: int, levels: int) -> float:
    """Relative solve cost of a nest: transforms of size (2n)^2 per level plus
    m^2 phase transforms per cross-level pair (Sec. 2.2: m transforms per axis)."""
    c = float(levels)
    for s in range(levels):
        for t in range(levels):
            if s != t:
                c += float(4 ** abs(s - t))
    return c * (2 * n) ** 2


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (1 rank: itself)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
