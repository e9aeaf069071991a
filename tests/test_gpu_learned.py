"""GPU parity of the learned-normal step (VOF_MIXED_LEARNED) against the
oracle's learned step, through the C ABI.

The networks here are built from their definition, not trained on the GPU:
the Youngs network (exact BF16 weights that make the network compute the
Youngs gradient), optionally with seeded random weights on every other unit,
and the all-zero network (no finite normal: MYC everywhere).  Bar: max |dc|
<= 1e-5 per cell and total volume within 1e-6 relative after one step.
Where the fallback decision lies within the oracle's ambiguity margin of
its threshold, both branches are valid; the GPU field must then match,
cell by cell, the oracle step that resolves the ambiguous decisions one way
or the other.
"""
import numpy as np
import pytest

import oracle as O
from helpers import youngs_network
from paper_2407_07463_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL32 = 1e-5


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


@pytest.fixture(scope="module")
def case():
    w = synth.make_workload("learned parity", shape=(36, 40, 44), phi=0.15, radius=5.0, n_modes=8,
                            amplitude=0.5, drift=1.0, cfl=0.3, seed=11)
    c = w.c.astype(np.float32).astype(np.float64)
    u = w.u.astype(np.float32).astype(np.float64)
    return c, u, w.dt


def gpu_step(vof, c, u, dt, params, tol, steps=1, step0=0):
    K, nz, ny, nx = c.shape
    cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=K, precision=2, tag_tau=0.0)
    c_d = torch.from_numpy(c).to(DEV, torch.float32).contiguous()
    u_d = torch.from_numpy(u).to(DEV, torch.float32).contiguous()
    ctx = vof.Context(cfg, c_d, u_d)
    wts = vof.vof_mlp_params_to_weights(torch.from_numpy(params.astype(np.float32)).to(DEV))
    ctx.vof_set_mlp(wts, tol)
    rep = ctx.vof_step(dt, steps)
    torch.cuda.synchronize()
    got = c_d.cpu().numpy().astype(np.float64)
    ctx.close()
    return got, rep


def p32(p):
    return p.astype(np.float32).astype(np.float64)


def test_learned_without_weights_is_a_state_error(vof, case):
    c, u, dt = case
    K, nz, ny, nx = c.shape
    cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=K, precision=2)
    c_d = torch.from_numpy(c).to(DEV, torch.float32).contiguous()
    u_d = torch.from_numpy(u).to(DEV, torch.float32).contiguous()
    ctx = vof.Context(cfg, c_d, u_d)
    with pytest.raises(vof.VofError) as e:
        ctx.vof_step(dt, 1)
    assert e.value.status == vof.VOF_ERR_STATE
    with pytest.raises(vof.VofError):
        ctx.vof_set_mlp(torch.zeros(vof.lib().vof_mlp_weights_size(), dtype=torch.uint8, device=DEV), -1.0)
    ctx.close()


def test_null_network_equals_mixed_myc_step(vof, case):
    """All-zero weights: every face falls back to MYC; the result is the
    oracle's plain step within the mixed-precision bar."""
    c, u, dt = case
    got, rep = gpu_step(vof, c, u, dt, np.zeros(O.MLP_NPARAM), 1e-3)
    want, _ = O.advect(c, u, dt, 1.0, 1)
    assert np.abs(got - want).max() <= TOL32
    assert rep["faces_network"] == 0 and rep["faces_myc"] > 0


def test_network_kept_everywhere_matches_oracle(vof, case):
    """Tolerance +inf (huge): the network's normal is used on every face,
    so no decision is taken and the step compares element by element."""
    c, u, dt = case
    p = p32(youngs_network(0.02, seed=3))
    got, rep = gpu_step(vof, c, u, dt, p, 1e30)
    want, _, counts = O.advect_step_learned(c, u, dt, 1.0, 0, p, tol=1e30, amb_eps=0.0)
    assert counts[1] == 0 and rep["faces_myc"] == 0
    err = np.abs(got - want).max()
    assert err <= TOL32, err
    assert abs(got.sum() - want.sum()) / want.sum() <= 1e-6
    # the listed faces are the oracle's interfacial donors, up to cells that
    # FP32 rounding leaves just inside (0, 1) in the later sweeps
    assert abs(rep["faces_network"] - counts[0]) <= 1e-2 * counts[0]


def stencils_of(cf):
    """Float stencils [n][27] of the interfacial cells of one periodic field,
    st[(dk+1)*9 + (dj+1)*3 + (di+1)] = c(i+di, j+dj, k+dk)."""
    planes = [np.roll(cf, shift=(-dk, -dj, -di), axis=(0, 1, 2))
              for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    S = np.stack(planes, -1)
    return S[(cf > 0) & (cf < 1)]


@pytest.mark.parametrize("tol", [1e-3, 0.0])
def test_judged_normals_match_oracle(vof, case, tol):
    """Per stencil (no propagation between decisions): the GPU's judged
    normal and its branch equal the oracle's wherever the oracle's residual
    lies outside the ambiguity margin of its threshold; inside it the GPU's
    normal is one of the two branches' normals."""
    c, _, _ = case
    st = np.concatenate([stencils_of(c[f]) for f in range(c.shape[0])]).astype(np.float32)
    st = st[np.random.default_rng(0).permutation(len(st))[:4000]]
    p = p32(youngs_network(0.02, seed=3))
    wts = vof.vof_mlp_params_to_weights(torch.from_numpy(p.astype(np.float32)).to(DEV))
    m, which = vof.vof_learned_normals(wts, torch.from_numpy(st).to(DEV), tol)
    m, which = m.cpu().numpy().astype(np.float64), which.cpu().numpy()
    eps, n_amb = 3e-5, 0
    for r in range(len(st)):
        s64 = st[r].astype(np.float64)
        ma, wa, amb = O.learned_normal(p, s64, tol, eps, 0)
        if amb:
            mb, _, _ = O.learned_normal(p, s64, tol, eps, 1)
            n_amb += 1
            assert min(np.abs(m[r] - ma).max(), np.abs(m[r] - mb).max()) <= 1e-4, r
        else:
            assert which[r] == wa, r
            assert np.abs(m[r] - ma).max() <= 1e-4, (r, m[r], ma)
    assert 0 < which.sum() < len(st)
    print("stencils", len(st), "network", int((which == 0).sum()), "ambiguous", n_amb)


def test_learned_step_with_fallback_against_oracle(vof):
    """Both branches within one step: a large sphere (radius 16 in 40^3,
    solenoidal flow), the perturbed Youngs network, tolerance 1e-3.

    The 27-cell mean residual that judges the network has near-ties: planes
    whose normals differ by 0.01-0.02 can explain a curved stencil with
    residuals equal to 1e-5, so some decisions fall inside the ambiguity
    margin (both branches valid) and their effects spread over the sweeps.
    What is unique is compared: every cell farther than four cells
    (Chebyshev, periodic; two per later sweep) from both cells of each face
    whose ambiguous decision changes the flux matches the oracle within 1e-5,
    and the total volume matches within 1e-6 relative."""
    shape = (40, 40, 40)
    c = synth.sphere_cell_fractions(shape, np.array([[19.6, 20.3, 19.9]]), 16.0)[None]
    c = c.astype(np.float32).astype(np.float64)
    u = synth.solenoidal_velocity(shape, 8, 0.5, 1.0, 5).astype(np.float32).astype(np.float64)
    dt = synth.dt_for_cfl(u, 0.3)
    tol = 1e-3
    p = p32(youngs_network(0.02, seed=3))
    got, rep = gpu_step(vof, c, u, dt, p, tol)
    amb = np.zeros(c.shape, dtype=np.uint8)
    want, _, counts = O.advect_step_learned(c, u, dt, 1.0, 0, p, tol=tol, amb_eps=3e-5, amb_map=amb)
    assert abs(got.sum() - want.sum()) / want.sum() <= 1e-6
    grown = amb.astype(bool)
    for ax in (1, 2, 3):
        g = grown.copy()
        for sft in range(-4, 5):
            if sft:
                g |= np.roll(grown, sft, axis=ax)
        grown = g
    changed = np.abs(want - c) > 0
    cmp = changed & ~grown
    print("faces", counts, "cells compared", int(cmp.sum()), "of", int(changed.sum()), "changed")
    assert cmp.sum() >= 1000
    err = np.abs(got - want)[~grown]
    assert err.max() <= TOL32, err.max()
    assert rep["faces_network"] > 1000 and rep["faces_myc"] > 1000


def test_trained_network_step_conserves_and_bounds(vof):
    """A network trained on the GPU, on the 256^3-like flow at small size:
    volume conserved to the mixed bar and c stays in [0, 1]."""
    tp = vof.train_params(n_train=1_000_000, n_test=10_000, epochs=2, batch=16384, seed=9)
    wts, _ = vof.vof_mlp_train(tp, DEV)
    w = synth.make_workload("learned trained", shape=(48, 48, 48), phi=0.2, radius=6.0, n_modes=8,
                            amplitude=0.5, drift=1.0, cfl=0.3, seed=12)
    K, nz, ny, nx = w.c.shape
    cfg = vof.make_config(nx, ny, nz, k_capacity=K, k_active=K, precision=2, tag_tau=0.0)
    c_d = torch.from_numpy(w.c).to(DEV, torch.float32).contiguous()
    u_d = torch.from_numpy(w.u).to(DEV, torch.float32).contiguous()
    v0 = c_d.double().sum().item()
    ctx = vof.Context(cfg, c_d, u_d)
    ctx.vof_set_mlp(wts, 1e-3)
    rep = ctx.vof_step(w.dt, 5)
    torch.cuda.synchronize()
    v1 = c_d.double().sum().item()
    assert abs(v1 + rep["clipped_volume"] - v0) / v0 <= 1e-6
    assert float(c_d.min()) >= 0.0 and float(c_d.max()) <= 1.0
    print(rep)
    assert rep["faces_network"] > 0 and rep["faces_myc"] > 0
    ctx.close()
