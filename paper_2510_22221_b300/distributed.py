"""Host logic of runs over several GPUs, one process per GPU (torchrun): the
partition of a batch's instances over the ranks and the whole-job rate.
There is no collective on the data path: every rank advances its own grids.
"""
from __future__ import annotations

import heapq


def shard_instances(cells, world: int) -> list:
    """Instance indices per rank, balanced by cell count: largest instance
    first onto the least-loaded rank (ties to the lower rank), each rank's
    list in increasing index order.  Deterministic for given cells and world."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda q: (-int(cells[q]), q))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for q in order:
        load, r = heapq.heappop(heap)
        out[r].append(q)
        heapq.heappush(heap, (load + int(cells[q]), r))
    return [sorted(s) for s in out]


def job_rate(units_local: float, seconds_local: float, group=None):
    """(units of all ranks / slowest rank's time, slowest rank's time) over the
    default process group (one rank: the local values)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return units_local / seconds_local, seconds_local
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / float(t.item()), float(t.item())
