"""The tagging entry point that allocates nothing (vof_label_noalloc).

It serves callers that cannot allocate device memory when they need drop
tags -- for example a plug-in whose host framework owns all device memory,
or a loop whose memory budget is fixed at start-up -- by keeping its scratch
in a fixed array inside the library.  Its tags must equal those of the
ordinary context-based vof_label, call after call: the scratch keeps the
previous call's contents, so the cases below run large grids before small
ones and the worst-case layout of the bit words (rows of at most 32 cells,
one word per row) at the maximum size.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


def ctx_labels(vof, c, precision, conn, tau):
    nz, ny, nx = c.shape
    cfg = vof.make_config(nx, ny, nz, k_capacity=1, k_active=1, precision=precision, connectivity=conn,
                          tag_tau=tau)
    u = torch.zeros((3, nz, ny, nx), dtype=c.dtype, device=c.device)
    ctx = vof.Context(cfg, c[None].contiguous(), u)
    lab, n = ctx.vof_label(0)
    out = lab.clone()
    ctx.close()
    return out, n


def field(rng, shape, density, tau=0.0):
    c = rng.random(shape) * (rng.random(shape) < density)
    if tau > 0.0:
        # cells exactly at the threshold as the float path sees it: a cell
        # holding float32(tau) is occupied iff float32(tau) > tau in double
        sel = rng.random(shape) < 0.05
        c[sel] = float(np.float32(tau))
    return c


def check(vof, c, precision, conn, tau):
    dt = torch.float64 if precision == 0 else torch.float32
    cd = torch.from_numpy(c).to("cuda", dt).contiguous()
    got, n = vof.vof_label_noalloc(cd, precision=precision, tag_tau=tau, connectivity=conn)
    want, nw = ctx_labels(vof, cd, precision, conn, tau)
    assert n == nw
    assert torch.equal(got, want)
    return n


@pytest.mark.parametrize("precision,conn", [(0, 6), (1, 26), (2, 6)])
def test_noalloc_matches_vof_label_twice(vof, precision, conn):
    rng = np.random.default_rng(7 + precision)
    # the largest grid first, then a smaller one over its leftover scratch
    for call, shape in enumerate([(64, 64, 64), (28, 36, 40)]):
        assert check(vof, field(rng, shape, 0.12 if call == 0 else 0.3), precision, conn, 0.0) > 0


@pytest.mark.parametrize("precision", [1, 2])
def test_noalloc_threshold_in_float(vof, precision):
    """tau = 0.1 with cells holding float32(0.1) (just above 0.1 in double):
    the float comparison must take the double decision, call after call."""
    rng = np.random.default_rng(21 + precision)
    for shape in [(40, 48, 56), (20, 24, 28)]:
        check(vof, field(rng, shape, 0.4, tau=0.1), precision, 6, 0.1)


def test_noalloc_short_rows_at_maximum_size(vof):
    """262144 cells in rows of 8 (one bit word per row: the most words the
    scratch holds), then a small grid, then the maximum grid again."""
    rng = np.random.default_rng(5)
    for shape, conn in [((64, 512, 8), 6), ((9, 10, 11), 26), ((64, 512, 8), 26)]:
        check(vof, field(rng, shape, 0.35), 0, conn, 0.0)


def test_noalloc_rejects_oversize(vof):
    c = torch.zeros((65, 64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(vof.VofError) as e:
        vof.vof_label_noalloc(c)
    assert e.value.status == -9
