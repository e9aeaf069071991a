"""Multi-process host logic of weak scaling over gloo (world size 2, CPU):
the timing reduction (max of the times, sum of the work), the
deterministic partition of independent boxes over ranks, and the reduction
of the drop statistics of every rank's boxes."""
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


def fake_stats(r):
    """A vof_stats-shaped result for rank r."""
    import numpy as np

    rng = np.random.default_rng(10 + r)
    Rm = rng.normal(size=(3, 3))
    Rm = Rm @ Rm.T
    return {"n_drops": 5 + 3 * r, "volume": 40.0 + 7.0 * r, "events": 2.0 + r, "M": rng.normal(size=3),
            "R": Rm, "chi_mean": 1.1 + 0.2 * r, "chi_max": 1.5 + r, "chi_drops": 4.0 + r,
            "hist_r": rng.integers(0, 5, size=6).astype(float),
            "hist_rt": rng.integers(0, 5, size=(6, 4)).astype(float)}


def stats_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = scaling.reduce_stats(fake_stats(rank), 1000.0 * (rank + 1))
    finally:
        dist.destroy_process_group()


def test_statistics_reduced_over_two_ranks():
    """The union of two ranks' boxes: counts, volumes and histograms add,
    moments are event-weighted, chi_mean drop-weighted, chi_max the larger;
    both ranks get the same result."""
    import numpy as np

    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(stats_worker, args=(2, port, out), nprocs=2, join=True)
    a, b = fake_stats(0), fake_stats(1)
    for g in (out[0], out[1]):
        assert g["n_drops"] == 13 and g["volume"] == pytest.approx(87.0) and g["events"] == pytest.approx(5.0)
        E = a["events"] + b["events"]
        np.testing.assert_allclose(g["M"], (a["events"] * a["M"] + b["events"] * b["M"]) / E, rtol=1e-14)
        Rg = (a["events"] * a["R"] + b["events"] * b["R"]) / E
        np.testing.assert_allclose(g["R"], Rg, rtol=1e-14)
        np.testing.assert_allclose(g["A"], Rg - np.trace(Rg) / 3 * np.eye(3), rtol=1e-13, atol=1e-15)
        assert g["chi_mean"] == pytest.approx((1.1 * 4 + 1.3 * 5) / 9)
        assert g["chi_max"] == 2.5 and g["chi_drops"] == 9.0
        assert g["d"] == pytest.approx((6 * (87.0 / 13) / np.pi) ** (1 / 3))
        assert g["n_p"] == pytest.approx(13 / 3000.0)
        np.testing.assert_array_equal(g["hist_r"], a["hist_r"] + b["hist_r"])
        np.testing.assert_array_equal(g["hist_rt"], a["hist_rt"] + b["hist_rt"])


def test_batched_boxes_split_over_ranks():
    """Each rank builds only its share of the batch, and a box is the same
    whichever others are built."""
    import numpy as np

    from paper_2407_07463_gb300 import synth

    specs = synth.batched_specs(seed=7, n_boxes=6, sizes=(16, 24))
    parts = scaling.partition(scaling.box_costs(specs), 2)
    assert sorted(parts[0] + parts[1]) == list(range(6))
    full = synth.config_batched(seed=7, n_boxes=6, sizes=(16, 24))
    for p in parts:
        sub = synth.config_batched(seed=7, n_boxes=6, sizes=(16, 24), select=set(p))
        assert len(sub) == len(p)
        for i, w in zip(sorted(p), sub):
            assert w.name == full[i].name and w.k_active == full[i].k_active
            np.testing.assert_array_equal(w.c, full[i].c)
            np.testing.assert_array_equal(w.u, full[i].u)
