"""Several GPUs: the spaces of a batch are independent, so they are sharded
across ranks with no collective on the data path; only the timings and
counts are reduced at the end (max of times, sum of work)."""
from __future__ import annotations

import heapq


def shard_lpt(costs, world: int):
    """Longest-processing-time-first assignment of jobs to ``world`` ranks.
    Returns a list of job-index lists, one per rank (deterministic)."""
    order = sorted(range(len(costs)), key=lambda j: (-costs[j], j))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for j in order:
        load, r = heapq.heappop(heap)
        out[r].append(j)
        heapq.heappush(heap, (load + costs[j], r))
    return [sorted(x) for x in out]


def reduce_time_work(ms: float, units: float, group=None, device="cpu"):
    """(max over ranks of ms, sum over ranks of units) through torch.distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
