#!/usr/bin/env python
"""Benchmark of one multi-field VoF time step (arXiv 2407.07463, Section 2.3).

A step is the whole hot path on one box: three split PLIC advection sweeps of
every active colour field, then the no-coalescence Steps 1-4 (near-contact
test on every field, tagging and recolouring when it fires).  The workload is
256^3 cells, K = 8 colour fields, phi = 0.3 (2347 spheres of radius 8 cells,
coloured greedily over the fields), a 16-mode solenoidal velocity with
amplitude 0.5 plus a vertical drift of 1, CFL 0.3.  Metric: cell-field updates
per second = cells x active fields x steps / time.  The headline path is FP32
with the learned normal (network trained on the GPU before the timed region,
MYC fallback); the plain FP64 path runs on the same workload for the ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank advances its own independent box (weak scaling) and
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VoF cell-field updates/s at 256^3 K=8; FP32+learned vs plain FP64 same GPU"
UNIT = "cell-field updates/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM = 6800.0
TAG_TAU = 1e-6  # occupancy threshold of Steps 1-4 (the library's default)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=256, help="cells per axis")
    p.add_argument("--k", type=int, default=8, help="colour fields")
    p.add_argument("--phi", type=float, default=0.3)
    p.add_argument("--precision", choices=["learned", "mixed", "fp64"], default="learned")
    p.add_argument("--train-samples", type=int, default=10_000_000)
    p.add_argument("--train-epochs", type=int, default=4)
    p.add_argument("--fp64-steps", type=int, default=3, help="steps of the FP64 comparison run")
    p.add_argument("--e2e-steps", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=64, help="sub-box edge of the reference arm's sample")
    p.add_argument("--workload", choices=["box", "batched", "nt"], default="box",
                   help="box: 256^3 K=8 (the headline); batched: 64 uneven boxes in one launch per pass; "
                        "nt: the tracer-count study N(t) over phi")
    p.add_argument("--boxes", type=int, default=64)
    p.add_argument("--no-batched", action="store_true", help="skip the 64-box batch extra key")
    return p.parse_args()


def workload(n, k, phi, seed):
    from paper_2407_07463_gb300 import synth

    return synth.make_workload(f"{n}^3 K={k} phi={phi} r=8", n=n, k_capacity=k, phi=phi, radius=8.0,
                               n_modes=16, amplitude=0.5, drift=1.0, cfl=0.3, steps=100, seed=seed)


def workload_desc(wl):
    return (f"{wl.shape[2]}^3 tri-periodic grid, K={wl.k_capacity} colour fields "
            f"({wl.k_active} active at t=0), {len(wl.centres)} spheres r=8 cells "
            f"(phi={wl.c.sum() / np.prod(wl.shape):.3f}), 16-mode solenoidal velocity amp 0.5 + "
            f"vertical drift 1, CFL 0.3, near-contact w=2 + recolouring every step")


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler is running (its first
            # line), so that the samples fall inside it
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- helpers


def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2407_07463_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM, "fallback 6.8 TB/s"


def algorithmic_bytes(cls, n_cells, fields, es):
    """Minimum DRAM bytes one launch of a kernel class must move.
    update (one sweep of every active field): read c_in and write c_out per
    cell-field, one c_c bit read or written and (last sweep) one occupancy
    bit per cell-field, the sweep's and the next sweep's velocity component
    per cell.  list_faces: read c per cell-field plus one velocity
    component.  pack_bits: read c per cell-field, write one bit.
    near_contact: read and write one bit per cell-field."""
    if cls == "update":
        return n_cells * fields * (2 * es + 2 / 8) + 2 * n_cells * es
    if cls == "list_faces":
        return n_cells * fields * es + n_cells * es
    if cls == "pack_bits":
        return n_cells * fields * (es + 1 / 8)
    if cls == "near_contact":
        return n_cells * fields * 2 / 8
    return None


# FP32 operations per listed face of the judged learned flux (counted from
# the kernel's formulation: the branch-free volume takes about 57 operations
# per cell, a plane constant about 100): the network normal's 27-cell
# residual with its plane constant, the plane's flux; for the faces above the
# tolerance also MYC's normal and residual.
RESIDUAL_FLOPS = 27 * 57 + 100
MYC_FLOPS = 120
FLUX_FLOPS = 60
# multiply-adds of the network per stencil (27-64-64-3), as algorithmic work
MLP_FLOPS = 2 * (27 * 64 + 64 * 64 + 64 * 3)


def bf16_peak():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s"


def sweep_bytes(n_cells, fields, es):
    """Algorithmic bytes of one sweep launch: the method's own minimum per
    step (read and write c once per cell-field, the three velocity
    components once per cell: 2 es + 3 es / K per cell-field update, 9.5 B
    at K = 8 in FP32) over the three sweeps of the step."""
    return step_bytes(n_cells, fields, es) / 3.0


def class_roofline(name, cnt, tot_ms, n_cells, fields, es, hbm, peak_src, launches_per_step):
    """HBM roofline entry of one kernel class from its live CUDA-event time:
    the units one launch processes (a sweep kernel: one sweep of every
    cell-field of the step) times the algorithmic bytes per unit, over the
    average launch duration."""
    avg_s = tot_ms / cnt * 1e-3
    if launches_per_step == 3:
        alg = sweep_bytes(n_cells, fields, es)
    else:
        alg = algorithmic_bytes(name, n_cells, fields, es)
        if alg is None:
            return None
    ach = alg / avg_s / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "algorithmic_bytes_per_launch": alg, "peak_source": peak_src}


def alu_roofline(cnt, tot_ms, rep, sm_count, sm_mhz):
    """FP32-issue view of the judged learned flux (an extra key): operations
    counted from the kernel's formulation over the FP32 lanes of the SMs."""
    faces = (rep.get("faces_network", 0) or 0) + (rep.get("faces_myc", 0) or 0)
    if not faces:
        return None
    avg_s = tot_ms / cnt * 1e-3
    per_launch = faces / cnt
    judged = (rep.get("faces_myc_judged", 0) or 0) / cnt
    flops = per_launch * (RESIDUAL_FLOPS + FLUX_FLOPS) + judged * (MYC_FLOPS + RESIDUAL_FLOPS)
    peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    ach = flops / avg_s / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "algorithmic_flops_per_launch": flops,
            "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (median SM clock)"}


def tensor_roofline(cnt, tot_ms, rep):
    faces = (rep.get("faces_network", 0) or 0) + (rep.get("faces_myc", 0) or 0)
    if not faces:
        return None
    flops = faces / cnt * MLP_FLOPS
    pk, src = bf16_peak()
    ach = flops / (tot_ms / cnt * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "algorithmic_flops_per_launch": flops, "peak_source": src}


def step_bytes(n_cells, fields, es):
    """The method's own minimum per step (read and write c once per step,
    the three velocity components once)."""
    return n_cells * fields * 2 * es + 3 * n_cells * es


def train_network(vof, torch, dev, args):
    """Network of the learned normal, trained on the GPU (untimed)."""
    tp = vof.train_params(n_train=args.train_samples, n_test=200_000, epochs=args.train_epochs,
                          batch=16384, seed=12345)
    t0 = time.perf_counter()
    w, rep = vof.vof_mlp_train(tp, dev)
    torch.cuda.synchronize()
    rep["seconds"] = time.perf_counter() - t0
    return w, rep


def host_network(seed=12345):
    """He-initialised weights of the same architecture (for the oracle's
    sample when no trained network is at hand; the oracle evaluates both
    estimators and both residuals on every donor, so its cost hardly depends
    on the weights)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(7312)
    p[0:2048].reshape(64, 32)[:, :27] = rng.normal(scale=math.sqrt(2 / 27), size=(64, 27))
    p[2048:6144] = rng.normal(scale=math.sqrt(2 / 64), size=4096)
    p[6144:7168].reshape(16, 64)[:3] = rng.normal(scale=math.sqrt(1 / 64), size=(3, 64))
    return p


def oracle_sample(c, u, dt, h, k_capacity, params, steps=1, omp=False, first_step=0):
    """The oracle as it stands on a sub-box: per step one advection step of
    every active field (learned normal with MYC fallback when params is not
    None, else MYC), then Steps 1-4.  omp: its OpenMP build over every core
    this process may use (z-planes of the advection in parallel; the rest is
    serial).  Returns (updates/s, seconds, updates, threads)."""
    import oracle

    oracle.build()
    threads = 1
    if omp:
        threads = oracle.threads(len(os.sched_getaffinity(0)))
    na = c.shape[0]
    t0 = time.perf_counter()
    for s in range(steps):
        if params is not None:
            c, _, _ = oracle.advect_step_learned(c, u, dt, h, first_step + s, params, tol=1e-3, omp=omp)
        else:
            c, _ = oracle.advect_step(c, u, dt, h, first_step + s, omp=omp)
        full = np.zeros((k_capacity,) + c.shape[1:])
        full[:na] = c[:na]
        full, na, _, _, _ = oracle.recolour(full, na, w=2, tau=TAG_TAU)
        c = full[:na]
    sec = time.perf_counter() - t0
    updates = int(np.prod(u.shape[1:])) * sum([c.shape[0]] * steps)
    return updates / sec, sec, updates, threads


def sub_box(wl, edge):
    return (np.ascontiguousarray(wl.c[:wl.k_active, :edge, :edge, :edge]),
            np.ascontiguousarray(wl.u[:, :edge, :edge, :edge]))


def oracle_sample_child(wl, edge, params, omp):
    """oracle_sample in a child process (the GPU process keeps its own
    threading runtime to itself); the inputs travel in a temporary file."""
    import tempfile

    c, u = sub_box(wl, edge)
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "sample.npz")
        np.savez(f, c=c, u=u, dt=wl.dt, h=wl.h, k=wl.k_capacity,
                 params=params if params is not None else np.zeros(0))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", f]
                           + (["--oracle-omp"] if omp else []), capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_main(path, omp):
    d = np.load(path)
    params = d["params"] if d["params"].size else None
    rate, sec, upd, thr = oracle_sample(d["c"], d["u"], float(d["dt"]), float(d["h"]), int(d["k"]), params,
                                        omp=omp)
    print(json.dumps({"rate": rate, "seconds": sec, "updates": upd, "threads": thr}))


def cpu_baseline(wl, params, learned):
    """The oracle timed on this machine's cores: the OpenMP build over every
    core on a 96^3 sub-box (the reported value) and the serial build on a
    48^3 sub-box, each one step of every active field plus Steps 1-4."""
    kind = "learned-normal" if learned else "MYC"
    res = {}
    for omp, edge in ((True, min(96, wl.shape[0])), (False, min(48, wl.shape[0]))):
        try:
            r = oracle_sample_child(wl, edge, params, omp)
        except (subprocess.CalledProcessError, OSError, ValueError) as e:
            res[omp] = {"error": str(e)[:200]}
            continue
        res[omp] = {"value": r["rate"], "unit": UNIT, "cores": r["threads"], "kind": "oracle",
                    "sample": f"one oracle step ({kind} advection, {'OpenMP over the z-planes' if omp else 'serial'}"
                              f", then Steps 1-4 serial) of the {edge}^3 sub-box, {wl.k_active} active fields "
                              f"({r['seconds']:.1f} s)"}
    out = dict(res[True]) if "value" in res[True] else dict(res[False])
    out["single_thread"] = res[False]
    out["cores_available"] = len(os.sched_getaffinity(0))
    return out


# --------------------------------------------------------------------------- reference arm


def run_reference(args, rank, world):
    """The oracle as it stands on this machine's cores (OpenMP build), on
    bounded sub-box samples of our arm's workload, same metric."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    wl = workload(args.n, args.k, args.phi, seed=3)
    edge = min(args.cpu_sample, args.n)
    c, u = sub_box(wl, edge)
    params = host_network()
    for _ in range(args.warmup):
        oracle_sample(c, u, wl.dt, wl.h, wl.k_capacity, params, omp=True)
    times = []
    upd = 0
    thr = 1
    for s_ in range(args.steps):
        _, t, n_, thr = oracle_sample(c, u, wl.dt, wl.h, wl.k_capacity, params, omp=True)
        times.append(t)
        upd += n_
    total = sum(times)
    value = upd / total
    sample = (f"{edge}^3 x {wl.k_active} fields sub-box of the workload, one oracle step per timed step "
              f"(learned-normal advection with He-initialised weights and MYC fallback, OpenMP over the "
              f"z-planes; Steps 1-4 serial)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(wl), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm


def error_vs_fp64(vof, torch, dev, wl, ref, steps, wts, rbins):
    """Each FP32 path (MYC; learned when weights are given) advanced from
    the initial state by `steps` steps with Steps 1-4, against the FP64 path
    after the same steps (ref): max |dc| per cell-field, max |dC| of the
    colour sum C = sum_k c_k (independent of which field a drop was moved
    to), and the relative difference of the total volume."""
    nz, ny, nx = wl.shape
    out = {"steps": steps, "against": "plain FP64 GPU path (MYC), same steps from the same state"}
    runs = [("mixed_myc", vof.VOF_MIXED, None)]
    if wts is not None:
        runs.insert(0, ("learned", vof.VOF_MIXED_LEARNED, wts))
    for name, prec, w in runs:
        cfg = vof.make_config(nx, ny, nz, k_capacity=wl.k_capacity, k_active=wl.k_active, precision=prec,
                              recolour=1, stats_rbins=rbins, stats_dr=0.16)
        c = torch.from_numpy(wl.c).to(dev, torch.float32).contiguous()
        u = torch.from_numpy(wl.u).to(dev, torch.float32).contiguous()
        ctx = vof.Context(cfg, c, u)
        if w is not None:
            ctx.vof_set_mlp(w, 1e-3)
        ctx.vof_step(wl.dt, steps)
        torch.cuda.synchronize()
        ctx.close()
        got = c.cpu().numpy().astype(np.float64)
        del ctx, c, u
        torch.cuda.empty_cache()
        out[name] = {"max_abs_per_cell_field": float(np.abs(got - ref).max()),
                     "max_abs_colour_sum": float(np.abs(got.sum(0) - ref.sum(0)).max()),
                     "rel_total_volume": float(abs(got.sum() - ref.sum()) / ref.sum())}
    return out


def timed_steps(torch, ctx, dt, steps):
    st = ctx.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    rep = ctx.vof_step(dt, steps, report=True)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), rep


def run_ours(args, rank, world):
    import torch

    from paper_2407_07463_gb300 import vof

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = workload(args.n, args.k, args.phi, seed=3 + rank)
    nz, ny, nx = wl.shape
    N = nx * ny * nz
    prec = {"learned": vof.VOF_MIXED_LEARNED, "mixed": vof.VOF_MIXED, "fp64": vof.VOF_FP64}[args.precision]
    tdt = torch.float64 if prec == vof.VOF_FP64 else torch.float32
    es = 8 if prec == vof.VOF_FP64 else 4
    train = None
    wts = None
    if prec == vof.VOF_MIXED_LEARNED:
        wts, train = train_network(vof, torch, dev, args)
    rbins = 2000
    cfg = vof.make_config(nx, ny, nz, k_capacity=wl.k_capacity, k_active=wl.k_active, precision=prec,
                          recolour=1, stats_rbins=rbins, stats_dr=0.16)
    c_d = torch.from_numpy(wl.c).to(dev, tdt).contiguous()
    u_d = torch.from_numpy(wl.u).to(dev, tdt).contiguous()
    ctx = vof.Context(cfg, c_d, u_d)
    if wts is not None:
        ctx.vof_set_mlp(wts, 1e-3)
    torch.cuda.synchronize()
    if args.warmup:
        ctx.vof_step(wl.dt, args.warmup)
    torch.cuda.synchronize()

    # timed region (launch timer on; barrier + synchronize on both sides)
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    ctx.vof_profile_enable(True)
    ctx.vof_profile_read()
    if dist:
        dist.barrier()
    sampler.start()
    l0 = ctx.launches
    ms, rep = timed_steps(torch, ctx, wl.dt, args.steps)
    launches = ctx.launches - l0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = ctx.vof_profile_read()
    ctx.vof_profile_enable(False)
    updates = N * rep["field_steps"]
    from paper_2407_07463_gb300 import scaling

    ms_max, updates_all = scaling.aggregate(ms, updates, device=dev)
    value = updates_all / (ms_max * 1e-3)

    # drop statistics (Section 3, Appendix A) of the state the timed steps
    # left, one event per rank, reduced over every rank's box
    stats = None
    try:
        st_ = ctx.vof_stats(reset=True, histograms=True)
        g_ = scaling.reduce_stats(st_, float(N) * cfg.h ** 3, device=dev)
        stats = {k: g_[k] for k in ("n_drops", "d", "n_p", "volume", "events", "chi_mean", "chi_max")}
        stats["A_zz"] = float(g_["A"][2, 2])
        stats["ranks"] = world
    except Exception as ex:  # reported, not fatal to the headline line
        stats = {"error": str(ex)[:200]}

    # the surface-tension source of the state the timed steps left (curvature
    # of every active field by height functions, then f = sum_i gamma kappa_i
    # grad C_i on the faces): algorithmic bytes = read c and write kappa per
    # cell-field, read c and kappa per cell-field, write f (3 per cell)
    st_extra = None
    try:
        f_out = torch.empty((3, nz, ny, nx), dtype=tdt, device=dev)
        ctx.vof_surface_tension(1.0, f_out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(ctx.stream)
        for _ in range(reps):
            ctx.vof_surface_tension(1.0, f_out)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        st_ms = e0.elapsed_time(e1) / reps
        na_ = rep["n_active"]
        alg = N * na_ * 4 * es + 3 * N * es
        hbm_, _ = peaks()
        st_extra = {"ms": st_ms, "fields": na_, "algorithmic_bytes": alg,
                    "achieved_gbs": alg / (st_ms * 1e-3) / 1e9, "frac_of_hbm": alg / (st_ms * 1e-3) / 1e9 / hbm_,
                    "what": "height-function curvature of every active field + surface-tension source on the faces"}
        del f_out
    except Exception as ex:  # reported, not fatal to the headline line
        st_extra = {"error": str(ex)[:200]}

    # e2e through the public API with host buffers: per step, pinned H2D of
    # the step's inputs (c and u), the step, D2H of the result (c).  Two
    # contexts on two streams take the steps in turn, so that the copies of
    # one overlap the step of the other (a stream of independent problems,
    # as a user would feed it); every copy is inside the timed region.
    e2e = None
    if args.e2e_steps > 0:
        c_h = torch.from_numpy(wl.c).to(tdt).pin_memory()
        u_h = torch.from_numpy(wl.u).to(tdt).pin_memory()
        pipe = []
        for _ in range(2):
            s_ = torch.cuda.Stream(device=dev)
            cd_ = torch.empty_like(c_d)
            ud_ = torch.empty_like(u_d)
            with torch.cuda.stream(s_):
                cd_.copy_(c_h, non_blocking=True)
                ud_.copy_(u_h, non_blocking=True)
            x_ = vof.Context(cfg, cd_, ud_, stream=s_)
            if wts is not None:
                x_.vof_set_mlp(wts, 1e-3)
            pipe.append((x_, s_, cd_, ud_, torch.empty_like(c_h).pin_memory()))
        fields0 = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(pipe[0][1])
        pipe[1][1].wait_event(e0)

        def upload(p_):
            with torch.cuda.stream(p_[1]):
                p_[2].copy_(c_h, non_blocking=True)
                p_[3].copy_(u_h, non_blocking=True)

        upload(pipe[0])
        for i in range(args.e2e_steps):
            cur, nxt = pipe[i % 2], pipe[(i + 1) % 2]
            if i + 1 < args.e2e_steps:
                upload(nxt)  # the next step's inputs travel during this step
            r = cur[0].vof_step(wl.dt, 1, report=True)
            fields0.append(r["field_steps"])
            with torch.cuda.stream(cur[1]):
                cur[4].copy_(cur[2], non_blocking=True)
        done = torch.cuda.Event()
        done.record(pipe[1][1])
        pipe[0][1].wait_event(done)
        e1.record(pipe[0][1])
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        for p_ in pipe:
            p_[0].close()
        e2e = {"value": N * sum(fields0) / (ems * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(c_h.numel() * es + u_h.numel() * es),
               "d2h_bytes_per_step": int(c_h.numel() * es), "steps": args.e2e_steps,
               "pipeline": "2 contexts on 2 streams: the copies of one step overlap the next step"}

    # FP64 comparison path on the same workload (plain FP64 kernels), and the
    # error of each reduced-precision result against it: every path starts
    # from the workload's initial state and takes the same steps (with
    # Steps 1-4), untimed
    fp64 = None
    err = None
    if not args.no_fp64 and prec != vof.VOF_FP64 and args.fp64_steps > 0:
        del ctx
        torch.cuda.empty_cache()
        cfg64 = vof.make_config(nx, ny, nz, k_capacity=wl.k_capacity, k_active=wl.k_active,
                                precision=vof.VOF_FP64, recolour=1, stats_rbins=rbins, stats_dr=0.16)
        c64 = torch.from_numpy(wl.c).to(dev).contiguous()
        u64 = torch.from_numpy(wl.u).to(dev).contiguous()
        ctx64 = vof.Context(cfg64, c64, u64)
        ctx64.vof_step(wl.dt, 1)
        ms64, rep64 = timed_steps(torch, ctx64, wl.dt, args.fp64_steps)
        fp64 = {"value": N * rep64["field_steps"] / (ms64 * 1e-3), "unit": UNIT,
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps}
        ctx64.close()
        ref = c64.cpu().numpy()
        del ctx64, c64, u64
        torch.cuda.empty_cache()
        err = error_vs_fp64(vof, torch, dev, wl, ref, 1 + args.fp64_steps, wts, rbins)

    # the 64-box batch (FP32 + learned, then FP64), untimed by the headline
    batched = None
    if not args.no_batched and prec == vof.VOF_MIXED_LEARNED:
        try:
            batched = batched_measure(vof, torch, dev, wts, 5, 2, 2, n_boxes=args.boxes, rank=rank, world=world)
        except Exception as ex:  # reported, not fatal to the headline line
            batched = {"error": str(ex)[:200]}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel class against HBM with the method's own
    # bytes (the ALU and tensor views of the learned kernels as extras)
    hbm, peak_src = peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fields = rep["field_steps"] / max(args.steps, 1)
    traffic_tab = {}
    try:
        with open(TRAFFIC) as f:
            tr = json.load(f)
        if tr.get("source_hash") == src_hash():
            traffic_tab = tr.get("kernels", {})
    except (OSError, ValueError):
        pass
    roof = roof_update = roof_alu = roof_tc = None
    for name, (cnt, tot) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        per_step = round(cnt / max(args.steps, 1))
        r = class_roofline(name, cnt, tot, N, fields, es, hbm, peak_src, per_step)
        if r is None:
            continue
        r.update({"kernel": name, "launches": cnt, "avg_ms": tot / cnt, "share_of_timed": tot / ms,
                  "traffic": traffic_tab.get(name)})
        if roof is None:
            roof = r
        if name == "update":
            own = algorithmic_bytes("update", N, fields, es)
            roof_update = dict(r, algorithmic_bytes_per_launch=own, achieved=own / (tot / cnt * 1e-3) / 1e9,
                               basis="the update pass's own bytes per sweep (c in and out, bits, velocities)")
            roof_update["frac"] = roof_update["achieved"] / hbm
        if name == "face_flux" and prec == vof.VOF_MIXED_LEARNED:
            roof_alu = alu_roofline(cnt, tot, rep, sm_count, sm_mhz)
        if name == "net_normals":
            roof_tc = tensor_roofline(cnt, tot, rep)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        params = vof.mlp_weights_to_params(wts) if wts is not None else None
        cpu = cpu_baseline(wl, params, prec == vof.VOF_MIXED_LEARNED)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == vof.VOF_FP64 else "f32", "data": "synthetic",
            "config": {"workload": workload_desc(wl),
                       "precision": "fp64" if prec == vof.VOF_FP64 else
                       "mixed (f32, f64 alpha band 1e-3 and clip sums)",
                       "normals": "learned (MLP 27-64-64-3, BF16 tcgen05, MYC fallback tol 1e-3)"
                       if prec == vof.VOF_MIXED_LEARNED else "MYC",
                       "faces_network": rep.get("faces_network"), "faces_myc": rep.get("faces_myc"),
                       "faces_myc_judged": rep.get("faces_myc_judged"),
                       "training": train,
                       "step_bytes_min": step_bytes(N, rep["field_steps"] / max(args.steps, 1), es),
                       "l2": "inputs larger than L2 (fields "
                       f"{wl.k_capacity * N * es / 1e6:.0f} MB)",
                       "parallelism": f"{world} independent boxes" if world > 1 else "1 box",
                       "n_active_end": rep["n_active"], "drops_moved": rep["n_moved"],
                       "near_contact_steps": rep["near_contact_steps"]},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "roofline_update_pass": roof_update, "roofline_alu": roof_alu, "roofline_tensor": roof_tc,
            "cpu_baseline": cpu, "fp64_path": fp64, "error_vs_fp64": err, "curvature": st_extra, "drop_stats": stats,
            "batched": batched,
            "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}}
    if fp64:
        line["over_fp64"] = value / world / fp64["value"]
    line["step_roofline_frac"] = (step_bytes(N, rep["field_steps"] / max(args.steps, 1), es) /
                                  (ms_max / args.steps * 1e-3) / 1e9 / hbm)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_measure(vof, torch, dev, wts, steps, warmup, fp64_steps, seed=5, n_boxes=64, rank=0, world=1):
    """n_boxes independent boxes per GPU (edges from {32,48,64,96,128}, phi
    0.05-0.3, K 2-8) advanced as one batch: FP32 + learned normal, then
    plain FP64 on the same boxes; each with its HBM roofline on the method's
    own bytes (read and write c once per cell-field, the velocity once per
    cell, per step).  With several ranks the job is world * n_boxes boxes,
    split over the ranks by their n^3 K cost (longest first, to the least
    loaded rank); the time is the slowest rank's, the work the sum."""
    from paper_2407_07463_gb300 import scaling, synth

    n_all = n_boxes * world
    mine = scaling.partition(scaling.box_costs(synth.batched_specs(seed, n_all)), world)[rank]
    ws = synth.config_batched(seed=seed, n_boxes=n_all, select=set(mine))
    hbm, peak_src = peaks()
    res = {}
    for prec, name in ((vof.VOF_MIXED_LEARNED, "learned"), (vof.VOF_FP64, "fp64")):
        dt_ = torch.float64 if prec == vof.VOF_FP64 else torch.float32
        es_ = 8 if prec == vof.VOF_FP64 else 4
        cs = [torch.from_numpy(w.c).to(dev, dt_).contiguous() for w in ws]
        us = [torch.from_numpy(w.u).to(dev, dt_).contiguous() for w in ws]
        B = vof.Batch(list(zip(cs, us, [w.dt for w in ws])), precision=prec, k_active=[w.k_active for w in ws])
        if prec == vof.VOF_MIXED_LEARNED:
            B.set_mlp(wts, 1e-3)
        B.step(max(warmup, 1))
        torch.cuda.synchronize()
        n_st = steps if prec != vof.VOF_FP64 else max(1, min(steps, fp64_steps))
        st = B.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.step(n_st)
        e1.record(st)
        torch.cuda.synchronize()
        rep = B.report()
        alg = sum(int(np.prod(w.shape)) * (w.k_active * 2 * es_ + 3 * es_) for w in ws)
        ms, units = scaling.aggregate(e0.elapsed_time(e1), rep["cell_fields_per_step"] * n_st, device=dev)
        _, alg = scaling.aggregate(0.0, alg, device=dev)
        ach = alg / (ms / n_st * 1e-3) / 1e9
        res[name] = {"value": units / (ms * 1e-3), "ms_per_step": ms / n_st,
                     "steps": n_st, "cell_fields_per_step": units / n_st,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                  "algorithmic_bytes_per_step": alg, "peak_source": peak_src},
                     "update_launch_shape": [rep["update_warps"], rep["update_blocks_per_sm"]],
                     "tuned_candidates": rep["tune_candidates"], "graph_launches": rep["graph_launches"]}
        B.close()
        del cs, us
        torch.cuda.empty_cache()
    res["over_fp64"] = res["learned"]["value"] / res["fp64"]["value"]
    res["workload"] = (f"{n_all} tri-periodic boxes ({len(ws)} on rank {rank} of {world}), edges "
                       f"{sorted(set(w.shape[0] for w in ws))}, phi 0.05-0.3, "
                       f"K 2-8 (raised to the colouring's need), spheres r=4 (edge<64) / 8, 16-mode velocity amp 0.5 "
                       f"+ drift 1, CFL 0.3, no recolouring")
    return res


def run_batched(args, rank, world):
    """The 64-box batch as its own line (the default line carries it as the
    extra key `batched`)."""
    import torch

    from paper_2407_07463_gb300 import vof

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wts, train = train_network(vof, torch, dev, args)
    r = batched_measure(vof, torch, dev, wts, args.steps, args.warmup, args.fp64_steps, n_boxes=args.boxes,
                        rank=rank, world=world)
    lv = r["learned"]
    line = {"metric": "VoF cell-field updates/s, 64 batched boxes; FP32+learned vs plain FP64 same GPU",
            "value": lv["value"], "unit": UNIT, "n_gpus": world, "steps": lv["steps"], "warmup": args.warmup,
            "ms_per_step": lv["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "cell_fields_per_step": lv["cell_fields_per_step"],
                       "update_launch_shape": lv["update_launch_shape"], "tuned_candidates": lv["tuned_candidates"],
                       "graph_launches": lv["graph_launches"], "training": train},
            "roofline": lv["roofline"], "fp64_path": r["fp64"], "over_fp64": r["over_fp64"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_nt(args, rank, world):
    """Tracer count N(t) under the seeded flow: the synthetic analogue of the
    paper's N(t) figure (Section 2.3).  For phi in 0.01, 0.05, 0.1, 0.2, N_b =
    125 drops of diameter 20 cells (d / h = 20) in a box of edge
    d (N_b pi / (6 phi))^(1/3), coloured greedily, advanced in FP32 (MYC)
    with Steps 1-4 every step under the 16-mode velocity (amplitude 0.5,
    vertical drift 1, CFL 0.3); N(t) = fields holding a drop at each step's
    Step 1.  Not a throughput line: one JSON line of the curves' summaries.
    FP64 by default: the FP32 path's round-off residues reach the occupancy
    threshold (1e-6) and, with no surface tension to heal them, multiply
    into fragments that Step 4 keeps moving."""
    import torch

    from paper_2407_07463_gb300 import synth, vof

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    out = {"study": "tracer count N(t) vs phi under the seeded synthetic flow (analogue of the N(t) figure)",
           "steps": args.steps, "drops": 125, "d_cells": 20, "precision": args.precision, "cases": []}
    for phi in (0.01, 0.05, 0.1, 0.2):
        n = int(round(20.0 * (125 * math.pi / (6.0 * phi)) ** (1.0 / 3.0)))
        wl = synth.make_workload(f"N(t) phi={phi}", n=n, k_capacity=16, phi=None, n_spheres=125, radius=10.0,
                                 n_modes=16, amplitude=0.5, drift=1.0, cfl=0.3, seed=40 + int(phi * 100))
        prec = {"learned": vof.VOF_MIXED, "mixed": vof.VOF_MIXED, "fp64": vof.VOF_FP64}[args.precision]
        tdt = torch.float64 if prec == vof.VOF_FP64 else torch.float32
        cfg = vof.make_config(n, n, n, k_capacity=16, k_active=wl.k_active, precision=prec, recolour=1)
        c = torch.from_numpy(wl.c).to(dev, tdt).contiguous()
        u = torch.from_numpy(wl.u).to(dev, tdt).contiguous()
        ctx = vof.Context(cfg, c, u)
        series, moved, stop = [], 0, None
        t0 = time.perf_counter()
        for s_ in range(args.steps):
            try:
                r = ctx.vof_step(wl.dt, 1)
            except vof.VofError as e:  # the synthetic flow has no surface tension: drops
                stop = f"step {s_}: {e}"  # shred, and a fixed-capacity list can overflow
                break
            series.append(r["n_in_use"])
            moved += r["n_moved"]
        sec = time.perf_counter() - t0
        ctx.close()
        series = np.array(series)
        out["cases"].append({"phi": phi, "edge": n, "k_initial": wl.k_active, "steps_run": len(series),
                             "n_max": int(series.max()) if len(series) else None,
                             "n_mean": float(series.mean()) if len(series) else None,
                             "n_final": int(series[-1]) if len(series) else None, "drops_moved": moved,
                             "stopped": stop, "seconds": sec, "series_every_10": series[::10].tolist()})
        del c, u
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    if "--oracle-sample" in sys.argv:
        oracle_sample_main(sys.argv[sys.argv.index("--oracle-sample") + 1], "--oracle-omp" in sys.argv)
        return
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world)
        return
    if args.workload == "nt":
        run_nt(args, rank, world)
        return
    run_ours(args, rank, world)


if __name__ == "__main__":
    main()
