"""Multi-process host logic of weak scaling over gloo (world size 2, CPU):
the timing reduction (max of the times, sum of the work) and the
deterministic partition of independent boxes over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2407_07463_gb300 import scaling  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = scaling.rank_env()
        costs = [7, 3, 9, 1, 4, 4, 8, 2]
        mine = scaling.partition(costs, w)[r]
        units = sum(costs[i] for i in mine)
        ms = 10.0 + 5.0 * r
        out[r] = (scaling.aggregate(ms, units), mine)
    finally:
        dist.destroy_process_group()


def test_aggregate_and_partition_two_ranks():
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(worker, args=(2, port, out), nprocs=2, join=True)
    (agg0, p0), (agg1, p1) = out[0], out[1]
    assert agg0 == agg1 == (15.0, 38.0)
    assert sorted(p0 + p1) == list(range(8)) and not set(p0) & set(p1)
    loads = [sum([7, 3, 9, 1, 4, 4, 8, 2][i] for i in p) for p in (p0, p1)]
    assert abs(loads[0] - loads[1]) <= 1


def test_single_process_is_identity():
    assert scaling.aggregate(3.5, 10) == (3.5, 10.0)
    assert scaling.partition([1, 2, 3], 1) == [[0, 1, 2]]
