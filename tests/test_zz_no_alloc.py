"""The tagging entry point that allocates nothing (vof_label_noalloc).

It serves callers that cannot allocate device memory when they need drop
tags -- for example code running while a stream is captured into a CUDA
graph, or a plug-in whose host framework owns all device memory -- by keeping
its scratch in a fixed array inside the library.  Its tags must equal those
of the ordinary context-based vof_label, call after call (the scratch keeps
the previous call's contents).  This file is collected last on purpose.
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


def ctx_labels(vof, c, precision, conn):
    nz, ny, nx = c.shape
    cfg = vof.make_config(nx, ny, nz, k_capacity=1, k_active=1, precision=precision, connectivity=conn,
                          tag_tau=0.0)
    u = torch.zeros((3, nz, ny, nx), dtype=c.dtype, device=c.device)
    ctx = vof.Context(cfg, c[None].contiguous(), u)
    lab, n = ctx.vof_label(0)
    out = lab.clone()
    ctx.close()
    return out, n


@pytest.mark.parametrize("precision,conn", [(0, 6), (1, 26)])
def test_noalloc_matches_vof_label_twice(vof, precision, conn):
    rng = np.random.default_rng(7 + precision)
    dt = torch.float64 if precision == 0 else torch.float32
    shapes = [(28, 36, 40), (64, 64, 64)]  # the second is the maximum size
    for call, shape in enumerate(shapes):
        c = rng.random(shape) * (rng.random(shape) < (0.3 if call == 0 else 0.12))
        cd = torch.from_numpy(c).to("cuda", dt).contiguous()
        got, n = vof.vof_label_noalloc(cd, precision=precision, tag_tau=0.0, connectivity=conn)
        want, nw = ctx_labels(vof, cd, precision, conn)
        assert n == nw
        assert torch.equal(got, want)


def test_noalloc_rejects_oversize(vof):
    c = torch.zeros((65, 64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(vof.VofError) as e:
        vof.vof_label_noalloc(c)
    assert e.value.status == -9
