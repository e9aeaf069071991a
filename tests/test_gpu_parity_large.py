"""GPU parity at the workloads' own sizes, through the C ABI.

- The learned path (FP32 + the network trained on the GPU, tolerance 1e-3)
  on a 96^3 box of the benchmark's family (phi = 0.3, spheres of radius 8
  greedily coloured over 8 fields) against the oracle: per stencil, per
  single sweep (velocity along one axis: every cell not next to an
  ambiguous decision, elementwise at 1e-5) and per full step (cells out of
  reach of the ambiguous decisions).
- One FP64 step of the 128^3, K = 4, phi = 0.1 workload against the oracle
  at 1e-12 relative per cell (relative to max(c, 1e-3), see fp64_gate), then
  Steps 1-4 on the GPU's own field, bit-exact against the oracle's.
- The 256^3, K = 8 benchmark workload itself, learned (velocity along one
  axis at a time) and FP64, advanced by the same launches the benchmark
  times; the oracle recomputes sampled windows.  A cell after one step depends only on cells within 4 of it per
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
# Margin of the fallback decision.  The judge compares two 27-cell mean
# residuals of order 1e-2.  Between the oracle (FP64 sums, FP64 network
# accumulation) and the GPU (FP32) they differ by the FP32 rounding of the
# 27-term sum (<= 27 u E ~ 5e-7 with u = 6e-8), of the plane constant
# (~1e-7 per cut cell, ~9 cells / 27) and of the network's normal (relative
# ~1e-6, moving each cut-cell volume by ~1e-6: <= 3e-7 on the mean) --
# together below 1e-6; decisions within twice that of the threshold may go
# either way.
AMB_EPS = 2e-6


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


@pytest.fixture(scope="module")
def box96():
    wl = synth.make_workload("96^3 learned parity", n=96, k_capacity=8, phi=0.3, radius=8.0, n_modes=16,
                             amplitude=0.5, drift=1.0, cfl=0.3, seed=3)
    return f32(wl.c[:wl.k_active]), f32(wl.u), wl.dt


def stencils_of(cf):
    """Stencils [n][27] of the interfacial cells of one periodic field."""
    planes = [np.roll(cf, shift=(-dk, -dj, -di), axis=(0, 1, 2))
              for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    S = np.stack(planes, -1)
    return S[(cf > 0) & (cf < 1)]


def test_trained_decisions_within_the_margin(vof, trained, box96):
    """Per stencil of the 96^3 box (no propagation): with the trained
    network, the GPU's branch and normal equal the oracle's wherever the
    oracle's residual is more than AMB_EPS from its threshold; the ambiguous
    ones are counted and reported."""
    w, params = trained
    c, _, _ = box96
    st = np.concatenate([stencils_of(c[f]) for f in range(c.shape[0])]).astype(np.float32)
    st = st[np.random.default_rng(0).permutation(len(st))[:20000]]
    m, which = vof.vof_learned_normals(w, torch.from_numpy(st).to(DEV), 1e-3)
    m, which = m.cpu().numpy().astype(np.float64), which.cpu().numpy()
    n_amb = n_diff = 0
    for r in range(len(st)):
        s64 = st[r].astype(np.float64)
        ma, wa, amb = O.learned_normal(params, s64, 1e-3, AMB_EPS, 0)
        if amb:
            # either branch is valid: the GPU's normal is one of the two
            mb, _, _ = O.learned_normal(params, s64, 1e-3, AMB_EPS, 1)
            n_amb += 1
            n_diff += int(np.abs(ma - mb).max() > 1e-4)
            assert min(np.abs(m[r] - ma).max(), np.abs(m[r] - mb).max()) <= 1e-4, r
            continue
        assert which[r] == wa, r
        assert np.abs(m[r] - ma).max() <= 1e-4, (r, m[r], ma)
    print(f"trained decisions: {len(st)} stencils, network {int((which == 0).sum())}, ambiguous {n_amb} "
          f"(of which the two branches' normals differ: {n_diff})")


def one_axis(u, axis):
    """The velocity with only its component along `axis`: the step's other
    two sweeps move nothing, so each listed face's flux reaches the final
    field unchanged and an ambiguous decision can affect only its own two
    cells."""
    v = np.zeros_like(u)
    v[axis] = u[axis]
    return v


def ambiguous_cells(amb):
    return amb.astype(bool)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_learned_sweep_96cube_trained_network(vof, trained, box96, axis):
    """One step with the velocity along one axis only (one active sweep),
    the GPU-trained network at tolerance 1e-3: every cell that no ambiguous
    decision touches matches the oracle within 1e-5."""
    w, params = trained
    c, u, dt = box96
    u = one_axis(u, axis)
    ctx, c_d, rep = gpu_advance(vof, c, u, dt, 2, weights=w, tol=1e-3)
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    amb = np.zeros(c.shape, dtype=np.uint8)
    want, _, counts = O.advect_step_learned(c, u, dt, 1.0, 0, params, tol=1e-3, amb_eps=AMB_EPS, amb_map=amb,
                                            omp=True)
    print("axis", axis, "GPU faces network/MYC", rep["faces_network"], rep["faces_myc"], "oracle", counts)
    share, ncmp = compare_learned(got, want, ambiguous_cells(amb), c, f"96^3 sweep along {axis}")
    assert ncmp >= 0.5 * int((np.abs(want - c) > 0).sum())
    # one-axis flow is compressible (the c_c term changes the volume); both
    # sides change it alike
    assert abs(got.sum() - want.sum()) / want.sum() <= 1e-6
    assert rep["faces_network"] > 0 and rep["faces_myc"] > 0


def test_learned_step_96cube_trained_network(vof, trained, box96):
    """The full three-sweep step: cells out of reach of every ambiguous
    decision match within 1e-5 (the reach is reported: a decision near its
    threshold spreads over up to 4 cells per axis in the later sweeps, and
    with this network near-ties are common, so few cells remain), the total
    volume within 1e-6 and c stays in [0, 1]."""
    w, params = trained
    c, u, dt = box96
    ctx, c_d, rep = gpu_advance(vof, c, u, dt, 2, weights=w, tol=1e-3)
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    amb = np.zeros(c.shape, dtype=np.uint8)
    want, _, counts = O.advect_step_learned(c, u, dt, 1.0, 0, params, tol=1e-3, amb_eps=AMB_EPS,
                                            amb_map=amb, omp=True)
    print("GPU faces network/MYC", rep["faces_network"], rep["faces_myc"], "oracle", counts)
    compare_learned(got, want, reach(amb), c, "96^3 learned")
    assert abs(got.sum() - want.sum()) / want.sum() <= 1e-6
    assert got.min() >= 0.0 and got.max() <= 1.0


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


@pytest.mark.parametrize("precision,axis", [(2, 0), (2, 1), (2, 2), (0, None)])
def test_bench_workload_256cube_sampled_windows(vof, trained, bench_workload, precision, axis):
    """The learned path runs with the velocity along one axis at a time (so
    that every ambiguous decision stays on its own two cells, see one_axis);
    the FP64 path with the full velocity."""
    wl = bench_workload
    w, params = trained
    na = wl.k_active
    if precision == 2:
        c, u = f32(wl.c), one_axis(f32(wl.u), axis)
    else:
        c, u = wl.c, wl.u
    ctx, c_d, rep = gpu_advance(vof, c, u, wl.dt, precision, weights=w if precision == 2 else None,
                                k_active=na)
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    # properties at full size: the FP64 step conserves the volume up to what
    # the clip removed; c stays in [0, 1]
    v0, v1 = c[:na].sum(), got[:na].sum()
    if precision == 0:  # the one-axis flows of the learned runs are compressible
        assert abs(v1 + rep["clipped_volume"] - v0) <= 1e-12 * v0
    assert got.min() >= 0.0 and got.max() <= 1.0
    rng = np.random.default_rng(17)
    size = INNER + 2 * MARGIN
    shares = []
    for q in range(6 if precision == 0 else 3):
        o = tuple(int(v) for v in rng.integers(0, 256, 3))
        cw = np.ascontiguousarray(crop(c[:na], o, size))
        uw = np.ascontiguousarray(crop(u, o, size))
        inner = (slice(None),) + (slice(MARGIN, MARGIN + INNER),) * 3
        gw = crop(got[:na], o, size)[inner]
        if precision == 2:
            amb = np.zeros(cw.shape, dtype=np.uint8)
            want, _, _ = O.advect_step_learned(cw, uw, wl.dt, 1.0, 0, params, tol=1e-3, amb_eps=AMB_EPS,
                                               amb_map=amb, omp=True)
            share, _ = compare_learned(gw, want[inner], ambiguous_cells(amb)[inner], cw[inner],
                                       f"256^3 window {o} (velocity along {axis})")
            shares.append(share)
        else:
            want, _ = O.advect_step(cw, uw, wl.dt, 1.0, 0, omp=True)
            fp64_gate(gw, want[inner])
    if shares:
        print("mean share of changed cells next to an ambiguous decision:", float(np.mean(shares)))
