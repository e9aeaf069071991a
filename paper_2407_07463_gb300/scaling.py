"""Host-side logic of multi-GPU runs: one process per GPU, each advancing
its own independent boxes (weak scaling, no data-path collective).  The
only exchange is the timing reduction at the end: the job time is the
slowest rank's, the work is the sum over ranks.  The functions take a
process group so that the same code runs over NCCL on GPUs and over gloo in
CPU tests."""
from __future__ import annotations

import os


def rank_env():
    """(rank, world_size, local_rank) of this process (torchrun variables)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(ms, units, device="cpu", group=None):
    """Max over ranks of the timed milliseconds and sum of the units
    (cell-field updates) processed; (ms, units) unchanged without a group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())


def partition(costs, world):
    """Deterministic assignment of independent units (boxes) to ranks:
    longest-processing-time first, each unit to the least loaded rank (ties
    to the lower rank).  Returns one list of unit indices per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]
