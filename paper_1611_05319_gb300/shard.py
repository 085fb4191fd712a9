"""Host-side sharding of independent frames across ranks (one process per GPU).

Frames never read one another, so a batch splits across GPUs with no exchange
in the data path.  ``lpt_partition`` balances the ranks by hole size (longest
processing time first: each frame, largest first, goes to the least-loaded
rank).  ``max_over_ranks`` and ``sum_over_ranks`` are the only collectives
(timing and counts, outside the data path): the step time of a job is the
slowest rank's, its pixel count the sum over the ranks.
"""
from __future__ import annotations

from typing import List, Sequence


def lpt_partition(weights: Sequence[int], world: int) -> List[List[int]]:
    """Indices of ``weights`` split into ``world`` lists with balanced sums
    (greedy LPT; ties go to the lowest rank, frames in index order within a rank)."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(weights)), key=lambda i: (-int(weights[i]), i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(weights[i])
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of ``value`` over the ranks of the default process group (identity
    without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def sum_over_ranks(value: int, dist=None, device=None) -> int:
    """Sum of the integer ``value`` over the ranks of the default process group
    (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return int(value)
    import torch
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t[0])
