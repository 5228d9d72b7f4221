"""Multi-GPU sharding of independent work (one process per GPU).

A single periodic box does not shard without domain decomposition, so N
processes run N independent replicas.  Boxes of a batch and requests of a
served stream are independent: they are partitioned over ranks with no
collective on the data path; only the final timing and counts are combined
(max of the elapsed times, sum of the units), on the host side of
torch.distributed.
"""

from __future__ import annotations


def shard_boxes(costs, rank: int, world: int) -> list[int]:
    """Indices of the boxes rank `rank` owns: longest-processing-time greedy
    assignment by cost (particles x steps), ties broken by index, so every
    rank computes the same partition without communicating."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    owner = [0] * len(costs)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += costs[k]
    return [k for k in range(len(costs)) if owner[k] == rank]


def shard_requests(n: int, rank: int, world: int) -> list[int]:
    """Round-robin assignment of a request stream in arrival order."""
    return list(range(rank, n, world))


def combine(units: float, seconds: float, dist=None, device=None) -> tuple[float, float]:
    """Whole-job (units, seconds): units summed over ranks, time = max over ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units, seconds
    import torch
    t = torch.tensor([units, seconds], dtype=torch.float64, device=device)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def gather_list(values: list, dist=None) -> list:
    """Concatenate per-rank lists on every rank (host objects)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(values))
    return [v for part in out for v in part]
