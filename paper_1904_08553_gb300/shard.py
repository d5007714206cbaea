"""Work split of the batched form over ranks (one process per GPU).

The graphs of the batched form are independent problems: a rank advances its
own share of them as one group, and no data crosses ranks during a step.  A
single temporal graph does not shard (its local-move passes would need a
label exchange every pass); for it, ranks run independent replicas.

Only host logic lives here: the partition, and the reductions of a rank's
timing and counters over the process group (any torch.distributed backend:
NCCL on GPUs, gloo on the CPU).
"""
from __future__ import annotations

import heapq
from typing import Sequence


def partition_graphs(cost: Sequence[int], world: int) -> list[list[int]]:
    """Greedy longest-processing-time split of graphs (cost: e.g. entries of
    each graph) over ``world`` ranks.  Returns each rank's graph indices in
    ascending order; every graph is in exactly one share, and the heaviest
    share exceeds the lightest by at most the largest single cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    shares: list[list[int]] = [[] for _ in range(world)]
    for g in sorted(range(len(cost)), key=lambda i: (-int(cost[i]), i)):
        load, r = heapq.heappop(heap)
        shares[r].append(g)
        heapq.heappush(heap, (load + int(cost[g]), r))
    return [sorted(s) for s in shares]


def _reduce(value: float, op_name: str, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    x = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=getattr(dist.ReduceOp, op_name))
    return float(x.item())


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    return _reduce(value, "MAX", device)


def sum_over_ranks(value: float, device=None) -> float:
    """Sum over the ranks (work units processed by the whole job)."""
    return _reduce(value, "SUM", device)
