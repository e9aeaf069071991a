"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

FP64 path: |c_gpu - c_oracle| <= 1e-12 per cell (volume fractions live in
[0, 1], so this is 1e-12 relative to the unit scale); labels, near-contact
flags and recolouring bit-exact on the GPU's own field.  Mixed path:
max |dc| <= 1e-5 per cell and total volume within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_07463_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


DEV = "cuda:0"


def make_case(shape, n_spheres, radius, seed, K=None, amp=0.5, drift=1.0, modes=6, cfl=0.3):
    cen = synth.rsa_centres(shape, radius, n_spheres, seed)
    col, used = synth.greedy_colours(shape, cen, radius, 2)
    K = K or int(used)
    if K < used:
        col = np.zeros_like(col)
    c = synth.coloured_fields(shape, cen, radius, col, K)
    u = synth.solenoidal_velocity(shape, modes, amp, drift, seed + 100)
    return c, u, synth.dt_for_cfl(u, cfl), int(used)


def run_gpu(vof, c, u, dt, steps, precision=0, k_active=None, **kw):
    kw.setdefault("tag_tau", 0.0)
    K, nz, ny, nx = c.shape
    dtp = torch.float64 if precision == 0 else torch.float32
    cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=k_active or K, precision=precision, **kw)
    c_d = torch.from_numpy(c).to(DEV, dtp).contiguous()
    u_d = torch.from_numpy(u).to(DEV, dtp).contiguous()
    ctx = vof.Context(cfg, c_d, u_d)
    rep = ctx.vof_step(dt, steps) if steps else None
    torch.cuda.synchronize()
    return ctx, c_d, u_d, rep


# ---------------------------------------------------------------- PLIC primitives


def random_normals(rng, n, degenerate=True):
    m = rng.normal(size=(n, 3))
    if degenerate:
        k = rng.integers(0, 3, size=n)
        z = rng.random(n) < 0.2
        m[z, k[z]] = 0.0
    return m / np.abs(m).sum(1, keepdims=True)


def test_plic_volume_and_alpha_fp64(vof):
    rng = np.random.default_rng(1)
    n = 4000
    m = random_normals(rng, n)
    c = rng.random(n)
    c[:200] = 10.0 ** rng.uniform(-14, -2, 200)
    c[200:400] = 1 - 10.0 ** rng.uniform(-14, -2, 200)
    md = torch.from_numpy(m).to(DEV)
    cd = torch.from_numpy(c).to(DEV)
    a = vof.vof_plic_alpha(md, cd).cpu().numpy()
    v = vof.vof_plic_volume(md, torch.from_numpy(a).to(DEV)).cpu().numpy()
    # the GPU's alpha reproduces c through the oracle's independent volume
    vo = np.array([O.plic_volume(m[t], a[t]) for t in range(n)])
    assert np.abs(vo - c).max() <= 1e-14
    assert np.abs(v - c).max() <= 1e-14
    # and the GPU volume equals the oracle's on arbitrary planes
    al = rng.uniform(-1, 1, n)
    vg = vof.vof_plic_volume(md, torch.from_numpy(al).to(DEV)).cpu().numpy()
    vo = np.array([O.plic_volume(m[t], al[t]) for t in range(n)])
    assert np.abs(vg - vo).max() <= 1e-14


def test_plic_alpha_mixed(vof):
    rng = np.random.default_rng(2)
    n = 4000
    m = random_normals(rng, n).astype(np.float32)
    c = rng.random(n).astype(np.float32)
    c[:300] = (10.0 ** rng.uniform(-7, -3, 300)).astype(np.float32)
    a = vof.vof_plic_alpha(torch.from_numpy(m).to(DEV), torch.from_numpy(c).to(DEV), precision=1,
                           band=1e-3).cpu().numpy()
    vo = np.array([O.plic_volume(m[t].astype(np.float64), float(a[t])) for t in range(n)])
    err = np.abs(vo - c.astype(np.float64))
    assert err.max() <= 2e-6


def test_plic_volume_fp32(vof):
    """FP32 volume (the piecewise closed form) against the oracle's volume of
    the same float inputs: arbitrary planes, including ones that miss the
    cube, normals with zero or tiny components, and unnormalised scales."""
    rng = np.random.default_rng(4)
    n = 20000
    m = random_normals(rng, n)
    k = rng.integers(0, 3, size=n)
    tiny = rng.random(n) < 0.1
    m[tiny, k[tiny]] *= 10.0 ** rng.uniform(-12, -3, tiny.sum())
    scale = np.where(np.arange(n) < n // 2, 1.0, 10.0 ** rng.uniform(-6, 3, n))
    m = (m * scale[:, None]).astype(np.float32)
    m64 = m.astype(np.float64)
    lo = np.minimum(m64, 0).sum(1)
    al = (lo + rng.uniform(-0.05, 1.05, n) * np.abs(m64).sum(1)).astype(np.float32)
    v = vof.vof_plic_volume(torch.from_numpy(m).to(DEV), torch.from_numpy(al).to(DEV), precision=1)
    v = v.cpu().numpy().astype(np.float64)
    vo = np.array([O.plic_volume(m64[t], float(al[t])) for t in range(n)])
    err = np.abs(v - vo)
    assert err.max() <= 1e-6, (err.max(), m[err.argmax()], al[err.argmax()])


# ---------------------------------------------------------------- normals


def test_normals_fp64(vof):
    c, u, dt, _ = make_case((20, 24, 28), 3, 4.0, seed=3, K=1)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 0)
    got = ctx.vof_normals(0).cpu().numpy()
    want = O.normals(c[0])
    assert np.abs(got - want).max() <= 1e-15
    ctx.close()


# ---------------------------------------------------------------- advection


@pytest.mark.parametrize("precision", [0, 1])
def test_steps_in_several_calls_equal_one_call(vof, precision):
    """Each call lists the first sweep's faces afresh (k_list_bx), along the
    step's rotated direction: three one-step calls (lists along x, y, z)
    end with the same bits as one three-step call (rows of 2 and 4 row
    chunks)."""
    c, u, dt, _ = make_case((20, 24, 256), 30, 4.0, seed=21)
    _, c_one, _, _ = run_gpu(vof, c, u, dt, 3, precision)
    ctx, c_many, _, _ = run_gpu(vof, c, u, dt, 0, precision)
    for _ in range(3):
        ctx.vof_step(dt, 1)
    torch.cuda.synchronize()
    assert np.array_equal(c_one.cpu().numpy(), c_many.cpu().numpy())
    ctx.close()


@pytest.mark.parametrize("shape,steps", [((32, 32, 32), 1), ((32, 32, 32), 20), ((28, 36, 40), 3),
                                         ((17, 23, 48), 2)])
def test_advect_fp64_matches_oracle(vof, shape, steps):
    n = 8 if shape == (32, 32, 32) else 4
    c, u, dt, _ = make_case(shape, n, 4.0, seed=sum(shape) + steps, K=None, cfl=0.25)
    ctx, c_d, _, rep = run_gpu(vof, c, u, dt, steps)
    want, clipped = O.advect(c, u, dt, 1.0, steps)
    got = c_d.cpu().numpy()
    err = np.abs(got - want).max()
    assert err <= TOL64, err
    assert rep["steps_done"] == steps
    assert abs(rep["clipped_volume"] - clipped.sum()) <= 1e-12
    ctx.close()


def test_advect_fp64_conservation(vof):
    c, u, dt, _ = make_case((40, 40, 40), 6, 5.0, seed=9, cfl=0.3)
    ctx, c_d, _, rep = run_gpu(vof, c, u, dt, 5)
    got = c_d.cpu().numpy()
    for f in range(c.shape[0]):
        assert abs(got[f].sum() + 0 - c[f].sum()) <= 1e-12 * c[f].sum() + abs(rep["clipped_volume"])
    ctx.close()


def test_advect_mixed_matches_oracle(vof):
    c, u, dt, _ = make_case((32, 40, 36), 6, 4.0, seed=5, cfl=0.3)
    c32 = c.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    ctx, c_d, _, rep = run_gpu(vof, c32, u32, dt, 1, precision=1)
    want, _ = O.advect(c32, u32, dt, 1.0, 1)
    got = c_d.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= TOL32
    rel = abs(got.sum() - want.sum()) / want.sum()
    assert rel <= 1e-6
    ctx.close()


@pytest.mark.parametrize("shape,steps", [((36, 40, 32), 3), ((33, 20, 70), 2), ((5, 12, 40), 3),
                                         ((64, 48, 48), 1)])
def test_fused_mixed_steps(vof, shape, steps):
    """The one-launch mixed step (ragged tiles, tiny z, every sweep order)
    against the FP64 oracle run on the same float-rounded inputs."""
    n = 6 if min(shape) > 8 else 3
    r = 4.0 if min(shape) > 8 else 2.0
    c, u, dt, _ = make_case(shape, n, r, seed=sum(shape) * 7 + steps, cfl=0.3)
    c32 = c.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    ctx, c_d, _, rep = run_gpu(vof, c32, u32, dt, steps, precision=1)
    want, clipped = O.advect(c32, u32, dt, 1.0, steps)
    got = c_d.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= TOL32
    assert abs(got.sum() - want.sum()) <= 1e-6 * want.sum()
    assert rep["field_steps"] == steps * c.shape[0]
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [(3, 5, 64), (9, 1, 96), (4, 6, 32), (2, 2, 128)])
def test_vectorised_rows_match_oracle(vof, precision, shape):
    """Rows of whole 32-cell words take the 16-byte-lane update: a partial
    last chunk, a single row per plane (the y neighbour is the cell itself),
    periodic wrap along x inside a warp, every sweep order."""
    c, u, dt, _ = make_case(shape, 2, 1.5, seed=sum(shape) + precision, cfl=0.3)
    if precision:
        c = c.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    ctx, c_d, _, rep = run_gpu(vof, c, u, dt, 3, precision=precision)
    want, clipped = O.advect(c, u, dt, 1.0, 3)
    got = c_d.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= (TOL64 if precision == 0 else TOL32)
    if precision == 0:
        assert abs(rep["clipped_volume"] - clipped.sum()) <= 1e-12
    ctx.close()


def test_fused_bits_feed_recolour(vof):
    """Step 1 after a fused step uses the occupancy bits the step wrote; the
    recolouring of the GPU's own field must equal the oracle's."""
    shape = (40, 40, 40)
    cen = synth.rsa_centres(shape, 4.0, 14, seed=48)
    c = synth.coloured_fields(shape, cen, 4.0, np.zeros(14, dtype=np.int64), 4)
    u = synth.solenoidal_velocity(shape, 8, 0.6, 0.5, 49)
    dt = synth.dt_for_cfl(u, 0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 0, precision=1, k_active=1, tag_tau=1e-6)
    na = 1
    for s in range(3):
        ctx.vof_step(dt, 1)
        adv = c_d.cpu().numpy().astype(np.float64)
        moved, na_g, st = ctx.vof_recolour()
        want, na, nm, st_o, _ = O.recolour(adv, na, tau=1e-6)
        assert (moved, na_g, st) == (nm, na, st_o)
        assert np.array_equal(c_d.cpu().numpy().astype(np.float64), want)
    ctx.close()


def test_plane_translation(vof):
    """A plane moved by u = (0,0,1) at CFL 1/4 for 4 steps is the initial
    field rolled by one cell (away from the seams of the non-periodic plane)."""
    from helpers import plane_field
    shape = (16, 10, 12)
    n = np.array([0.12, -0.08, 1.0])
    n /= np.abs(n).sum()
    c0 = plane_field(O, shape, n, (5.0, 5.0, 7.3))[None]
    u = synth.uniform_velocity(shape, (0.0, 0.0, 1.0))
    ctx, c_d, _, _ = run_gpu(vof, c0, u, 0.25, 4)
    got = c_d.cpu().numpy()[0]
    want = np.roll(c0[0], 1, axis=0)
    inner = (slice(None), slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(got[inner], want[inner], atol=1e-12, rtol=0)
    ctx.close()


def test_cfl_and_nonfinite_errors(vof):
    shape = (8, 8, 8)
    c = np.zeros((1,) + shape)
    u = synth.uniform_velocity(shape, (0.0, 0.0, 1.0))
    ctx, c_d, _, _ = run_gpu(vof, c, u, 0.1, 0)
    with pytest.raises(vof.VofError) as e:
        ctx.vof_step(0.6, 1)
    assert e.value.status == -5
    ctx.close()
    u[0, 1, 2, 3] = np.nan
    with pytest.raises(vof.VofError) as e:
        run_gpu(vof, c, u, 0.1, 0)
    assert e.value.status == -8


# ---------------------------------------------------------------- tagging and Steps 1-4


@pytest.mark.parametrize("conn", [6, 26])
@pytest.mark.parametrize("shape", [(16, 16, 32), (9, 13, 48), (5, 7, 70), (11, 3, 96), (40, 33, 64)])
def test_label_bit_exact(vof, shape, conn):
    rng = np.random.default_rng(sum(shape) + conn)
    c = rng.random(shape) * (rng.random(shape) < 0.35)
    ctx, c_d, _, _ = run_gpu(vof, c[None], np.zeros((3,) + shape), 0.0, 0, connectivity=conn)
    lab, n = ctx.vof_label(0)
    want, nw = O.label(c, 0.0, conn)
    assert n == nw
    assert np.array_equal(lab.cpu().numpy(), want)
    ctx.close()


def test_label_after_advection(vof):
    c, u, dt, _ = make_case((32, 32, 32), 8, 4.0, seed=21, K=1, cfl=0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 6)
    lab, n = ctx.vof_label(0)
    want, nw = O.label(c_d.cpu().numpy()[0])
    assert n == nw and np.array_equal(lab.cpu().numpy(), want)
    ctx.close()


def test_near_contact_flags(vof):
    rng = np.random.default_rng(7)
    shape = (12, 14, 40)
    K = 4
    c = rng.random((K,) + shape) * (rng.random((K,) + shape) < np.array([0.0, 0.002, 0.02, 0.2])[:, None, None, None])
    for w in (1, 2, 3):
        ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + shape), 0.0, 0, stencil_w=w)
        flags = ctx.vof_near_contact()
        for f in range(K):
            assert bool(flags[f]) == O.near_contact(c[f], w)
        ctx.close()


def criterion_panel(name):
    from test_oracle_tag import load_criterion_panel
    return load_criterion_panel(name)


def test_worked_example_on_gpu(vof):
    meta, ci, cj, centre = criterion_panel("left")
    c = np.zeros((3,) + ci.shape)
    c[0], c[1] = ci, cj
    ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + ci.shape), 0.0, 0, k_active=2)
    assert ctx.vof_near_contact()[0] == 1
    moved, na, st = ctx.vof_recolour()
    assert (moved, na, st) == (1, 3, 0)
    want, na_o, nm_o, st_o, _ = O.recolour(c, 2)
    assert np.array_equal(c_d.cpu().numpy(), want)
    ctx.close()
    meta, ci, cj, centre = criterion_panel("right")
    ctx, c_d, _, _ = run_gpu(vof, np.stack([ci[:], np.zeros_like(ci)]), np.zeros((3,) + ci.shape), 0.0, 0,
                             k_active=1)
    assert ctx.vof_near_contact()[0] == 1
    moved, na, st = ctx.vof_recolour()
    assert moved == 0 and na == 1
    ctx.close()


def cubes(rng, shape, K, n, size=3):
    c = np.zeros((K,) + shape)
    for _ in range(n):
        lo = [int(rng.integers(0, s)) for s in shape]
        sl = tuple(np.arange(l, l + size) % s for l, s in zip(lo, shape))
        c[0][np.ix_(*sl)] = rng.uniform(0.3, 1.0)
    return c


@pytest.mark.parametrize("seed", range(6))
def test_recolour_bit_exact(vof, seed):
    rng = np.random.default_rng(100 + seed)
    shape = (20, 18, 32) if seed % 2 else (16, 16, 16)
    K = 3 if seed < 3 else 6
    c = cubes(rng, shape, K, 6 + 2 * seed)
    want, na_o, nm_o, st_o, _ = O.recolour(c, 1)
    ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + shape), 0.0, 0, k_active=1)
    moved, na, st = ctx.vof_recolour()
    assert (moved, na, st) == (nm_o, na_o, st_o)
    assert np.array_equal(c_d.cpu().numpy(), want)
    ctx.close()


# Rows of 1, 2, 4 and 8 whole words, with partial tiles along y and z: the
# shared-memory tiles of Step 1 (256 / W rows a block, a halo of w rows).
TILED_SHAPES = [(20, 18, 32), (20, 13, 64), (12, 11, 128), (12, 9, 256)]


@pytest.mark.parametrize("shape", TILED_SHAPES)
@pytest.mark.parametrize("w", [1, 2, 3])
def test_near_contact_flags_tiled(vof, shape, w):
    """Step 1 on rows of whole words (the tiled kernel where the tile and its
    halo fit the grid) equals the oracle field by field."""
    rng = np.random.default_rng(sum(shape) * 10 + w)
    K = 10
    dens = np.array([0.0, 0.0001, 0.0003, 0.001, 0.05] + [0.0] * 5)[:, None, None, None]
    c = rng.random((K,) + shape) * (rng.random((K,) + shape) < dens)
    nz, ny, nx = shape
    # one pair per field around an empty middle cell: across a tile's edge
    # in y, across the periodic ends in y, z and x; then a pair three cells
    # apart (no middle cell)
    j1 = min(15, ny - 3)
    c[5, 8, j1, 31], c[5, 8, j1 + 2, 31] = 0.7, 0.6
    c[6, 0, ny - 1, 5], c[6, 0, 1, 5] = 0.5, 0.9
    c[7, nz - 1, 3, 9], c[7, 1, 3, 9] = 0.8, 0.4
    c[8, 2, 4, nx - 1], c[8, 2, 4, 1] = 0.6, 0.6
    c[9, 4, 6, 30], c[9, 4, 6, 33 % nx] = 0.9, 0.9
    ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + shape), 0.0, 0, stencil_w=w)
    flags = ctx.vof_near_contact()
    for f in range(K):
        assert bool(flags[f]) == O.near_contact(c[f], w), f
    ctx.close()


def cubes_in_fields(rng, shape, K, k_active, n, size=3):
    """n cubes of random fractions spread over the first k_active fields."""
    c = np.zeros((K,) + shape)
    for q in range(n):
        lo = [int(rng.integers(0, s)) for s in shape]
        sl = tuple(np.arange(l, l + size) % s for l, s in zip(lo, shape))
        c[q % k_active][np.ix_(*sl)] = rng.uniform(0.3, 1.0)
    return c


@pytest.mark.parametrize("shape,n,k_active", [((20, 18, 32), 40, 1), ((16, 12, 64), 40, 2),
                                              ((12, 11, 128), 60, 3), ((10, 12, 256), 80, 3)])
def test_recolour_bit_exact_whole_word_rows(vof, shape, n, k_active):
    """Steps 1-4 where the rows are whole words: tiled Step 1, every flagged
    field tagged in one chain (run-head links, tags written only where a
    word is occupied), pairs, the dilated touch test and the move -- the
    fields after the call equal the oracle's bit for bit."""
    rng = np.random.default_rng(sum(shape) + n)
    K = 8
    c = cubes_in_fields(rng, shape, K, k_active, n)
    want, na_o, nm_o, st_o, _ = O.recolour(c, k_active)
    ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + shape), 0.0, 0, k_active=k_active)
    moved, na, st = ctx.vof_recolour()
    assert (moved, na, st) == (nm_o, na_o, st_o)
    assert moved > 0
    assert np.array_equal(c_d.cpu().numpy(), want)
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_recolour_with_threshold(vof, precision):
    """tau = 1e-6: round-off residues below tau are not drops; the float path
    decides c > tau exactly as the double comparison does."""
    rng = np.random.default_rng(55 + precision)
    shape = (18, 20, 40)
    c = cubes(rng, shape, 4, 10)
    resid = (rng.random(shape) < 0.05) * 10.0 ** rng.uniform(-12, -4, shape)
    c[0] = np.where(c[0] == 0, resid, c[0])
    c[0][0, 0, :4] = [1e-6, np.nextafter(1e-6, 1), float(np.float32(1e-6)), 2e-6]
    if precision:
        c = c.astype(np.float32).astype(np.float64)
    want, na_o, nm_o, st_o, _ = O.recolour(c, 1, tau=1e-6)
    ctx, c_d, _, _ = run_gpu(vof, c, np.zeros((3,) + shape), 0.0, 0, precision=precision, k_active=1,
                             tag_tau=1e-6)
    lab, n = ctx.vof_label(0)
    lo, no = O.label(c[0], 1e-6)
    assert n == no and np.array_equal(lab.cpu().numpy(), lo)
    moved, na, st = ctx.vof_recolour()
    assert (moved, na, st) == (nm_o, na_o, st_o)
    assert np.array_equal(c_d.cpu().numpy().astype(np.float64), want)
    ctx.close()


def test_step_then_recolour_sequence(vof):
    """Advect-then-recolour for a few steps, K = 4: each advection matches the
    oracle within 1e-12 and each recolouring of the GPU's own field matches
    the oracle's recolouring of that field bit for bit."""
    shape = (40, 40, 40)
    cen = synth.rsa_centres(shape, 4.0, 12, seed=44)
    col = np.zeros(len(cen), dtype=np.int64)
    col[::2] = 1
    c = synth.coloured_fields(shape, cen, 4.0, col, 4)
    u = synth.solenoidal_velocity(shape, 8, 0.6, 0.5, 45)
    dt = synth.dt_for_cfl(u, 0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 0, k_active=2)
    prev = c.copy()
    na = 2
    for s in range(4):
        ctx.vof_step(dt, 1)
        adv = c_d.cpu().numpy()
        want, _ = O.advect_step(prev, u, dt, 1.0, s)
        assert np.abs(adv - want).max() <= TOL64
        moved, na_g, st = ctx.vof_recolour()
        want, na, nm, st_o, _ = O.recolour(adv, na)
        assert (moved, na_g, st) == (nm, na, st_o)
        prev = c_d.cpu().numpy()
        assert np.array_equal(prev, want)
    ctx.close()


def test_step_with_recolour_flag(vof):
    shape = (32, 32, 32)
    cen = synth.rsa_centres(shape, 4.0, 10, seed=46)
    c = synth.coloured_fields(shape, cen, 4.0, np.zeros(10, dtype=np.int64), 4)
    u = synth.solenoidal_velocity(shape, 8, 0.6, 0.5, 47)
    dt = synth.dt_for_cfl(u, 0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 0, k_active=1, recolour=1)
    rep = ctx.vof_step(dt, 3)
    got = c_d.cpu().numpy()
    assert rep["n_active"] >= 1 and rep["steps_done"] == 3
    for f in range(rep["n_active"]):
        lab, n = O.label(got[f])
        assert len(O.near_pairs(got[f], lab, 2)) == 0
    ctx.close()


@pytest.mark.parametrize("k_active", [1, 5])
def test_step_with_recolour_matches_oracle(vof, k_active):
    """Steps with Steps 1-4 inside one vof_step call equal the oracle's
    advect-then-recolour sequence: FP64 fields within 1e-12, the same drops
    moved.  With one active field the moves activate new fields (the face
    list is made again); with five they go to active fields, and the face
    list of the next step is rewritten for the moved drops."""
    shape = (32, 32, 32)
    cen = synth.rsa_centres(shape, 4.0, 14, seed=52)
    c = synth.coloured_fields(shape, cen, 4.0, np.zeros(len(cen), dtype=np.int64), 6)
    u = synth.solenoidal_velocity(shape, 8, 0.6, 0.5, 53)
    dt = synth.dt_for_cfl(u, 0.3)
    steps = 4
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 0, k_active=k_active, recolour=1)
    rep = ctx.vof_step(dt, steps)
    got = c_d.cpu().numpy()
    prev, na, moved = c.copy(), k_active, 0
    for s in range(steps):
        adv, _ = O.advect_step(prev, u, dt, 1.0, s)
        prev, na, nm, st_o, _ = O.recolour(adv, na)
        moved += nm
    print(f"moved {moved}, fields {na}")
    assert moved > 0 and rep["n_moved"] == moved and rep["n_active"] == na
    assert np.abs(got - prev).max() <= TOL64
    ctx.close()


# ---------------------------------------------------------------- statistics


def test_drop_table_and_pair_stats(vof):
    c, u, dt, _ = make_case((48, 48, 48), 14, 4.0, seed=31, K=None, cfl=0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 3, stats_rbins=400, stats_dr=0.08)
    got_c = c_d.cpu().numpy()
    cens = []
    for f in range(c.shape[0]):
        lab, n = ctx.vof_label(f)
        vol, cen = ctx.vof_drop_table(f, lab, n)
        lo, no = O.label(got_c[f])
        vo, co = O.drop_table(got_c[f], lo, no)
        assert n == no
        np.testing.assert_allclose(vol.cpu().numpy(), vo, rtol=1e-12, atol=0)
        cg = cen.cpu().numpy()
        d = cg - co
        d -= 48 * np.round(d / 48)
        assert np.abs(d).max() <= 1e-11
        cens.append(cg)
    cen_all = np.concatenate(cens)
    hr, hrt, mom = vof.vof_pair_stats(torch.from_numpy(cen_all).to(DEV), [48.0] * 3, 400, 0.08,
                                      tie_tol=1e-10)
    ps = O.PairStats(400, 0.08).add(cen_all, [48.0] * 3, tie_tol=1e-10)
    assert np.array_equal(hr.cpu().numpy(), ps.hist_r)
    assert np.array_equal(hrt.cpu().numpy(), ps.hist_rt)
    m = mom.cpu().numpy()
    np.testing.assert_allclose(m[:3], ps.msum, atol=1e-9)
    np.testing.assert_allclose(m[3:12], ps.rsum, rtol=1e-12)
    assert m[12] == ps.E
    st = ctx.vof_stats(reset=True)
    assert st["n_drops"] == len(cen_all)
    assert st["events"] == len(cen_all)
    ctx.close()


def test_state_roundtrip(vof):
    c, u, dt, _ = make_case((24, 24, 24), 3, 4.0, seed=61, K=None, cfl=0.3)
    ctx, c_d, _, _ = run_gpu(vof, c, u, dt, 2)
    blob = ctx.vof_get_state()
    ctx.vof_step(dt, 3)
    after = c_d.clone()
    ctx.vof_set_state(blob)
    ctx.vof_step(dt, 3)
    assert torch.equal(c_d, after)
    ctx.close()
