"""Sharding of independent local solves over ranks (one process per GPU).

Local reconstructions are independent (paper Sec. 5.5: they can be computed in parallel),
so the work splits by region with no exchange on the data path: each rank solves its own
share and only the timing is reduced.  Assignment is greedy longest-processing-time by
estimated cost (box pixels x angles x iterations), deterministic for a given input.
"""
from __future__ import annotations

import heapq
import math


def region_cost(region, iters: int, n_angles: int) -> float:
    """Work estimate of one solve: (box side)^2 x angles x iterations (box side 2 ceil(r + m))."""
    side = 2 * math.ceil(region[2] + region[3])
    return float(side * side) * n_angles * max(int(iters), 1)


def assign(costs, world: int):
    """Greedy LPT: items in decreasing cost go to the least-loaded rank (ties: lower rank).
    Returns a list of index lists, one per rank; every index appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max if seconds_max > 0 else 0.0
