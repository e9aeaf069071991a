"""Host-side logic of multi-GPU runs: one process per GPU, each advancing
its own independent boxes (weak scaling, no data-path collective).  The
exchanges happen after the timed steps: the timing reduction (the job time
is the slowest rank's, the work is the sum over ranks) and the reduction of
the drop statistics of all ranks' boxes.  The functions take a process
group so that the same code runs over NCCL on GPUs and over gloo in CPU
tests."""
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


def box_costs(specs):
    """Work estimate of each box of a batch from its (edge n, phi, K) spec:
    n^3 K cell-fields per step."""
    return [float(n) ** 3 * k for n, _phi, k in specs]


def reduce_stats(st, box_volume, device="cpu", group=None):
    """Drop statistics of the union of every rank's independent boxes, from
    this rank's `vof_stats` result `st` (its boxes' total volume L^3 in
    `box_volume`).  Counts, volumes, events and the pair histograms add; the
    moments M and R are event-weighted means and A = R - tr(R)/3 delta; the
    mean aspect ratio is weighted by the drops that entered it and its
    maximum is the largest; the equivalent diameter and the number density
    are taken from the totals.  Without a process group the totals are this
    rank's."""
    import math

    import numpy as np
    import torch
    import torch.distributed as dist

    E = float(st["events"])
    M = np.asarray(st["M"], dtype=np.float64).reshape(3)
    R = np.asarray(st["R"], dtype=np.float64).reshape(9)
    hr = st.get("hist_r")
    hrt = st.get("hist_rt")
    sums = np.concatenate([[float(st["n_drops"]), float(st["volume"]), E, float(box_volume),
                            float(st["chi_mean"]) * float(st["chi_drops"]), float(st["chi_drops"])],
                           E * M, E * R])
    parts = [sums]
    if hr is not None:
        parts += [np.asarray(hr, dtype=np.float64).ravel(), np.asarray(hrt, dtype=np.float64).ravel()]
    flat = np.concatenate(parts)
    chi_max = float(st["chi_max"])
    if dist.is_available() and dist.is_initialized():
        t = torch.from_numpy(flat).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        flat = t.cpu().numpy()
        m = torch.tensor([chi_max], dtype=torch.float64, device=device)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
        chi_max = float(m.item())
    n, vol, E, L3, chi_sum, chi_n = (float(v) for v in flat[:6])
    M = flat[6:9] / E if E > 0 else np.zeros(3)
    R = (flat[9:18] / E if E > 0 else np.zeros(9)).reshape(3, 3)
    out = {"n_drops": int(round(n)), "volume": vol, "events": E, "M": M, "R": R,
           "A": R - np.trace(R) / 3.0 * np.eye(3),
           "d": (6.0 * (vol / n) / math.pi) ** (1.0 / 3.0) if n > 0 else 0.0,
           "n_p": n / L3 if L3 > 0 else 0.0,
           "chi_mean": chi_sum / chi_n if chi_n > 0 else 0.0, "chi_max": chi_max, "chi_drops": chi_n}
    if hr is not None:
        nr = np.asarray(hr).size
        out["hist_r"] = flat[18:18 + nr]
        out["hist_rt"] = flat[18 + nr:].reshape(np.asarray(hrt).shape)
    return out
