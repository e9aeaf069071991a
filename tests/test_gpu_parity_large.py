"""GPU parity at the workloads' own sizes, through the C ABI.

- One learned step (FP32 + the network trained on the GPU, tolerance 1e-3)
  on a 96^3 box of the benchmark's family (phi = 0.3, spheres of radius 8
  greedily coloured over 8 fields) against the oracle's learned step,
  elementwise at 1e-5 outside the cells that ambiguous fallback decisions
  can reach.
- One FP64 step of the 128^3, K = 4, phi = 0.1 workload against the oracle
  at 1e-12 relative per cell (relative to max(c, 1e-3), see fp64_gate), then
  Steps 1-4 on the GPU's own field, bit-exact against the oracle's.
- The 256^3, K = 8 benchmark workload itself, learned and FP64, advanced by
  the same launches the benchmark times; the oracle recomputes sampled
  windows.  A cell after one step depends only on cells within 4 of it per
  axis (each sweep reads the 3x3x3 stencils of the donors on both faces:
  +-2 along its own axis, +-1 across), so the oracle's step on a periodic
  window with a 6-cell margin reproduces the window's interior exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_07463_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL32 = 1e-5
AMB_EPS = 3e-5


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    O.threads(0)
    return vof


@pytest.fixture(scope="module")
def trained(vof):
    """A network trained on the GPU by the library's own kernels (seeded,
    shorter than the benchmark's run), and its parameters for the oracle."""
    tp = vof.train_params(n_train=2_000_000, n_test=20_000, epochs=2, batch=16384, seed=31)
    w, rep = vof.vof_mlp_train(tp, DEV)
    torch.cuda.synchronize()
    print("training:", {k: rep[k] for k in ("final_loss", "test_mean_deg_mlp", "test_mean_deg_myc")})
    return w, vof.mlp_weights_to_params(w)


def f32(a):
    return a.astype(np.float32).astype(np.float64)


def gpu_advance(vof, c, u, dt, precision, steps=1, weights=None, tol=1e-3, **kw):
    K, nz, ny, nx = c.shape
    dtp = torch.float64 if precision == 0 else torch.float32
    cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=kw.pop("k_active", K), precision=precision,
                          **kw)
    c_d = torch.from_numpy(c).to(DEV, dtp).contiguous()
    u_d = torch.from_numpy(u).to(DEV, dtp).contiguous()
    ctx = vof.Context(cfg, c_d, u_d)
    if weights is not None:
        ctx.vof_set_mlp(weights, tol)
    rep = ctx.vof_step(dt, steps)
    torch.cuda.synchronize()
    return ctx, c_d, rep


def grow(mask, r, axes):
    out = mask.copy()
    for ax in axes:
        g = out.copy()
        for s in range(-r, r + 1):
            if s:
                g |= np.roll(out, s, axis=ax)
        out = g
    return out


def reach(amb):
    """Cells an ambiguous decision can affect: an ambiguous face changes the
    fluxes of its two cells, and the later sweeps of the step spread that by
    at most 2 cells per sweep (4 in all)."""
    return grow(amb.astype(bool), 4, (-3, -2, -1))


def compare_learned(got, want, grown, c0, tag):
    """Elementwise check outside the reach of the ambiguous decisions."""
    changed = np.abs(want - c0) > 0
    cmp = changed & ~grown
    share = float(grown[changed].mean()) if changed.any() else 0.0
    err = np.abs(got - want)[~grown]
    print(f"{tag}: changed cells {int(changed.sum())}, compared {int(cmp.sum())}, "
          f"share inside the ambiguity reach {share:.4f}, max |dc| outside {err.max():.3e}")
    assert err.max() <= TOL32, err.max()
    return share, int(cmp.sum())


def test_learned_step_96cube_trained_network(vof, trained):
    w, params = trained
    wl = synth.make_workload("96^3 learned parity", n=96, k_capacity=8, phi=0.3, radius=8.0, n_modes=16,
                             amplitude=0.5, drift=1.0, cfl=0.3, seed=3)
    c, u = f32(wl.c[:wl.k_active]), f32(wl.u)
    assert c.shape[0] >= 5
    ctx, c_d, rep = gpu_advance(vof, c, u, wl.dt, 2, weights=w, tol=1e-3)
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    amb = np.zeros(c.shape, dtype=np.uint8)
    want, _, counts = O.advect_step_learned(c, u, wl.dt, 1.0, 0, params, tol=1e-3, amb_eps=AMB_EPS,
                                            amb_map=amb, omp=True)
    print("GPU faces network/MYC", rep["faces_network"], rep["faces_myc"], "oracle", counts)
    share, ncmp = compare_learned(got, want, reach(amb), c, "96^3 learned")
    assert share <= 0.10 and ncmp >= 10000
    assert abs(got.sum() - want.sum()) / want.sum() <= 1e-6
    assert rep["faces_network"] > 0 and rep["faces_myc"] > 0


def fp64_gate(got, want):
    """The FP64 bar, 1e-12 relative per cell, read relative to max(c, 1e-3):
    cells holding at least 1e-3 of their volume are held to 1e-12 of their
    value; a smaller fraction is the difference of O(1) face fluxes and
    carries their absolute rounding, so it is held to 1e-15 absolute."""
    err = np.abs(got - want)
    scale = np.maximum(np.abs(want), 1e-3)
    worst = float((err / scale).max())
    print(f"FP64: max |dc| {err.max():.3e}, max |dc| / max(c, 1e-3) {worst:.3e}")
    assert worst <= 1e-12


def test_fp64_step_128cube_k4_then_steps_1_to_4(vof):
    wl = synth.config_medium()
    c, u = wl.c, wl.u
    K = wl.k_capacity
    ctx, c_d, rep = gpu_advance(vof, c, u, wl.dt, 0, k_active=wl.k_active, tag_tau=0.0)
    got = c_d.cpu().numpy()
    want, _ = O.advect_step(c, u, wl.dt, 1.0, 0, omp=True)
    fp64_gate(got, want)
    # Steps 1-4 on the GPU's own field against the oracle's
    n_moved, n_active, _ = ctx.vof_recolour()
    torch.cuda.synchronize()
    after = c_d.cpu().numpy()
    ctx.close()
    ref, na, nm, st, _ = O.recolour(got, wl.k_active, w=2, tau=0.0)
    assert (n_moved, n_active) == (nm, na)
    assert np.array_equal(after, ref)
    print("128^3 K=4: moved", nm, "active", na, "of", K)


@pytest.fixture(scope="module")
def bench_workload():
    return synth.make_workload("256^3 K=8 phi=0.3 r=8", n=256, k_capacity=8, phi=0.3, radius=8.0, n_modes=16,
                               amplitude=0.5, drift=1.0, cfl=0.3, steps=100, seed=3)


def crop(a, origin, size):
    """Periodic crop of the last three axes starting at origin (z, y, x)."""
    idx = [(np.arange(size) + o) % n for o, n in zip(origin, a.shape[-3:])]
    return a[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


MARGIN, INNER = 6, 24


@pytest.mark.parametrize("precision", [2, 0])
def test_bench_workload_256cube_sampled_windows(vof, trained, bench_workload, precision):
    wl = bench_workload
    w, params = trained
    na = wl.k_active
    if precision == 2:
        c, u = f32(wl.c), f32(wl.u)
    else:
        c, u = wl.c, wl.u
    ctx, c_d, rep = gpu_advance(vof, c, u, wl.dt, precision, weights=w if precision == 2 else None,
                                k_active=na)
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    # properties at full size: the clip removed nothing to speak of, every
    # field conserved its volume, c stays in [0, 1]
    v0, v1 = c[:na].sum(), got[:na].sum()
    assert abs(v1 + rep["clipped_volume"] - v0) <= (1e-6 if precision else 1e-12) * v0
    assert got.min() >= 0.0 and got.max() <= 1.0
    rng = np.random.default_rng(17)
    size = INNER + 2 * MARGIN
    shares = []
    for q in range(6):
        o = tuple(int(v) for v in rng.integers(0, 256, 3))
        cw = np.ascontiguousarray(crop(c[:na], o, size))
        uw = np.ascontiguousarray(crop(u, o, size))
        inner = (slice(None),) + (slice(MARGIN, MARGIN + INNER),) * 3
        gw = crop(got[:na], o, size)[inner]
        if precision == 2:
            amb = np.zeros(cw.shape, dtype=np.uint8)
            want, _, _ = O.advect_step_learned(cw, uw, wl.dt, 1.0, 0, params, tol=1e-3, amb_eps=AMB_EPS,
                                               amb_map=amb, omp=True)
            share, _ = compare_learned(gw, want[inner], reach(amb)[inner], cw[inner], f"256^3 window {o}")
            shares.append(share)
        else:
            want, _ = O.advect_step(cw, uw, wl.dt, 1.0, 0, omp=True)
            fp64_gate(gw, want[inner])
    if shares:
        assert np.mean(shares) <= 0.10
