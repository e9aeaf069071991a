"""Batched boxes (one launch per sweep pass for every box, graph replay,
tuned launch shape) against the same boxes advanced one by one through
their own contexts, and against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2407_07463_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


@pytest.fixture(scope="module")
def boxes():
    ws = synth.config_batched(seed=7, n_boxes=6, sizes=(32, 48, 64))
    # one non-cubic box with a partial row chunk and a single-row plane
    shape = (12, 1, 36)
    cen = synth.rsa_centres(shape, 2.0, 2, 3)
    col, used = synth.greedy_colours(shape, cen, 2.0, 2)
    c = synth.coloured_fields(shape, cen, 2.0, col, int(used))
    u = synth.solenoidal_velocity(shape, 4, 0.5, 1.0, 4)
    ws.append(synth.Workload("flat", shape, int(used), int(used), c, u, synth.dt_for_cfl(u, 0.3), 1.0, 1, 2.0,
                             cen, col))
    return ws


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt).contiguous()


def run_contexts(vof, ws, precision, steps, weights=None):
    dt_ = torch.float64 if precision == 0 else torch.float32
    out = []
    for w in ws:
        K, nz, ny, nx = w.c.shape
        cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=w.k_active, precision=precision,
                              tag_tau=1e-6)
        c_d, u_d = dev(w.c, dt_), dev(w.u, dt_)
        ctx = vof.Context(cfg, c_d, u_d)
        if weights is not None:
            ctx.vof_set_mlp(weights, 1e-3)
        ctx.vof_step(w.dt, steps)
        torch.cuda.synchronize()
        out.append(c_d.cpu().numpy())
        ctx.close()
    return out


def run_batch(vof, ws, precision, steps, weights=None, **kw):
    dt_ = torch.float64 if precision == 0 else torch.float32
    cs = [dev(w.c, dt_) for w in ws]
    us = [dev(w.u, dt_) for w in ws]
    B = vof.Batch(list(zip(cs, us, [w.dt for w in ws])), precision=precision, k_active=[w.k_active for w in ws],
                  **kw)
    if weights is not None:
        B.set_mlp(weights, 1e-3)
    B.step(steps)
    rep = B.report()
    torch.cuda.synchronize()
    out = [c.cpu().numpy() for c in cs]
    B.close()
    return out, rep


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_contexts(vof, boxes, precision):
    want = run_contexts(vof, boxes, precision, 4)
    got, rep = run_batch(vof, boxes, precision, 4)
    for b, (g, w) in enumerate(zip(got, want)):
        assert np.array_equal(g, w), b
    assert rep["steps_done"] == 4 and rep["graph_launches"] == 3 and rep["direct_steps"] == 1
    assert rep["tune_candidates"] > 1 and rep["update_blocks_per_sm"] >= 1


def test_batch_without_graph_or_tuning(vof, boxes):
    want = run_contexts(vof, boxes, 1, 2)
    got, rep = run_batch(vof, boxes, 1, 2, use_graph=False, autotune=False)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert rep["graph_launches"] == 0 and rep["tune_candidates"] == 0


def test_batch_learned_equals_contexts(vof, boxes):
    tp = vof.train_params(n_train=1_000_000, n_test=10_000, epochs=2, batch=16384, seed=3)
    wts, _ = vof.vof_mlp_train(tp, DEV)
    want = run_contexts(vof, boxes, 2, 3, weights=wts)
    got, rep = run_batch(vof, boxes, 2, 3, weights=wts)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert rep["faces_network"] > 0 and rep["faces_myc"] > 0


def test_batch_fp64_matches_oracle(vof, boxes):
    small = [w for w in boxes if w.c[0].size <= 48 ** 3][:3]
    got, rep = run_batch(vof, small, 0, 2)
    for g, w in zip(got, small):
        want, clipped = O.advect(w.c[:w.k_active], w.u, w.dt, 1.0, 2)
        assert np.abs(g[:w.k_active] - want).max() <= 1e-12
        assert np.array_equal(g[w.k_active:], w.c[w.k_active:])


def test_batch_argument_errors(vof, boxes):
    w = boxes[0]
    c = dev(w.c, torch.float32)
    u = dev(w.u, torch.float32)
    bad = dev(np.zeros((1, 8, 8, 10)), torch.float32)  # rows of 10 cells: not whole 16-byte lanes
    ub = dev(np.zeros((3, 8, 8, 10)), torch.float32)
    with pytest.raises(vof.VofError):
        vof.Batch([(bad, ub, 0.1)], precision=1)
    with pytest.raises(vof.VofError) as e:
        vof.Batch([(c, u, 10.0)], precision=1)  # CFL far above 1/2
    assert e.value.status == vof.VOF_ERR_CFL
    B = vof.Batch([(c, u, w.dt)], precision=2)
    with pytest.raises(vof.VofError) as e:
        B.step(1)
    assert e.value.status == vof.VOF_ERR_STATE
    B.close()
