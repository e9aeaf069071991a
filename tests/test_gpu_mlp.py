"""GPU parity of the learned normal estimator (tensor-core forward and
backward passes) against the FP64 oracle, and the gain of the trained network
over MYC on held-out stencils."""
import numpy as np
import pytest

import oracle as O

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


def bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("k,n", [(16, 16), (32, 64), (64, 64), (64, 16)])
def test_tensor_core_operand_layout(vof, k, n):
    rng = np.random.default_rng(k * n)
    A = rng.normal(size=(128, k)).astype(np.float32)
    B = rng.normal(size=(n, k)).astype(np.float32)
    d = vof.vof_tc_gemm_check(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)).cpu().numpy()
    want = bf16(A) @ bf16(B).T
    assert np.abs(d - want).max() <= 1e-5 * np.abs(want).max()


def test_bounded_wait_gives_up_and_device_stays_usable(vof):
    """A wait on an mbarrier that nothing arrives at returns VOF_ERR_TIMEOUT
    (no fault); the next tensor-core call still works."""
    assert vof.vof_wait_selftest(100000) == vof.VOF_ERR_TIMEOUT
    A = torch.ones((128, 16), device=DEV)
    B = torch.ones((16, 16), device=DEV)
    d = vof.vof_tc_gemm_check(A, B).cpu().numpy()
    assert np.all(d == 16.0)


def random_params(rng, scale=0.25):
    p = rng.normal(size=O.MLP_NPARAM) * scale
    p[0:2048].reshape(64, 32)[:, 27:] = 0.0          # W1 padding columns
    p[6144:7168].reshape(16, 64)[3:, :] = 0.0        # W3 padding rows
    p[7296 + 3:] = 0.0                               # b3 padding
    return p


def plane_stencils(rng, n):
    st = np.zeros((n, 27))
    tg = np.zeros((n, 3))
    for r in range(n):
        nv = rng.normal(size=3)
        nv /= np.linalg.norm(nv)
        a0 = rng.uniform(-0.49, 0.49) * np.abs(nv).sum()
        for k in (-1, 0, 1):
            for j in (-1, 0, 1):
                for i in (-1, 0, 1):
                    st[r, (k + 1) * 9 + (j + 1) * 3 + (i + 1)] = O.plic_volume(
                        nv, a0 - (nv[0] * (i - 0.5) + nv[1] * (j - 0.5) + nv[2] * (k - 0.5)))
        tg[r] = nv
    return st.astype(np.float32), tg.astype(np.float32)


def frame_is_ambiguous(st, rel=1e-5):
    """The canonical frame (reflections by the signs of the Youngs
    components, axes ordered by their magnitudes) can flip between FP32 and
    FP64 when two |components| agree, or one is zero, to within rounding."""
    y = np.abs(O.youngs(st.astype(np.float64).reshape(3, 3, 3)))
    ys = np.sort(y)
    scale = ys[-1] + 1e-300
    return ys[0] <= rel * scale or (ys[1] - ys[0]) <= rel * scale or (ys[2] - ys[1]) <= rel * scale


def test_mlp_forward_matches_oracle(vof):
    """Elementwise: each normal within 2e-5 of the oracle's (BF16 weights,
    (hi, lo) BF16 layer inputs, FP64 sums; the GPU sums in FP32), except
    stencils whose canonical frame sits on a rounding boundary -- counted,
    at most 1% of them, and those still within 2 degrees."""
    rng = np.random.default_rng(3)
    p = random_params(rng)
    w = vof.vof_mlp_params_to_weights(torch.from_numpy(p.astype(np.float32)).to(DEV))
    st, _ = plane_stencils(rng, 400)
    st += (rng.random(st.shape) < 0.1) * rng.normal(scale=0.05, size=st.shape).astype(np.float32)
    st = np.clip(st, 0, 1).astype(np.float32)
    got = vof.vof_mlp_forward(w, torch.from_numpy(st).to(DEV)).cpu().numpy().astype(np.float64)
    p32 = p.astype(np.float32).astype(np.float64)
    worst, boundary = 0.0, 0
    for r in range(len(st)):
        want = O.mlp_normal(p32, st[r].astype(np.float64).reshape(3, 3, 3), bf16=True)
        err = float(np.abs(got[r] - want).max())
        if frame_is_ambiguous(st[r]):
            boundary += 1
            assert np.degrees(np.arccos(np.clip(got[r] @ want, -1, 1))) < 2.0
            continue
        worst = max(worst, err)
        assert err <= 2e-5, (r, got[r], want)
    print("max elementwise error", worst, "frame-boundary stencils", boundary, "of", len(st))
    assert boundary <= 0.01 * len(st)


def test_mlp_gradients_match_oracle(vof):
    """GPU backward (tensor cores, BF16 operands) against FP64 backprop of the
    same BF16-rounded forward: relative L2 error <= 1e-2 per tensor."""
    rng = np.random.default_rng(4)
    p = random_params(rng)
    w = vof.vof_mlp_params_to_weights(torch.from_numpy(p.astype(np.float32)).to(DEV))
    st, tg = plane_stencils(rng, 512)
    g_gpu, loss_sum = vof.vof_mlp_grad(w, torch.from_numpy(st).to(DEV), torch.from_numpy(tg).to(DEV))
    g_gpu = g_gpu.cpu().numpy().astype(np.float64)
    xs, ts = [], []
    for r in range(len(st)):
        x, sg, pm = O.mlp_canon(st[r].astype(np.float64).reshape(3, 3, 3))
        xs.append(x)
        ts.append([sg[pm[q]] * tg[r][pm[q]] for q in range(3)])
    loss, g = O.mlp_loss_grad(p.astype(np.float32).astype(np.float64), np.array(xs), np.array(ts), bf16=True)
    assert loss_sum / len(st) == pytest.approx(loss, rel=1e-2)
    spans = {"W1": (0, 2048), "W2": (2048, 6144), "W3": (6144, 7168), "b1": (7168, 7232),
             "b2": (7232, 7296), "b3": (7296, 7312)}
    for name, (a, b) in spans.items():
        rel = np.linalg.norm(g_gpu[a:b] - g[a:b]) / max(np.linalg.norm(g[a:b]), 1e-30)
        assert rel <= 1e-2, (name, rel)


def test_training_gains_over_myc(vof):
    """Train on 4M generated stencils (planes and spheres); on held-out
    stencils the network's 95th-percentile angular error is below MYC's, and
    the estimator as the step uses it (network, MYC fallback when the
    network's plane explains the 3x3x3 block worse than MYC's and worse than
    1e-3) beats MYC on both the mean and the 95th percentile."""
    tp = vof.train_params(n_train=4_000_000, n_test=200_000, epochs=4, batch=16384, seed=7)
    w, rep = vof.vof_mlp_train(tp, DEV)
    print(rep)
    assert rep["final_loss"] < 1e-2
    assert rep["test_p95_deg_mlp"] < rep["test_p95_deg_myc"]
    assert rep["test_mean_deg_combined"] < rep["test_mean_deg_myc"]
    assert rep["test_p95_deg_combined"] < rep["test_p95_deg_myc"]
    # by class: the network's gain is on curved interfaces (sphere radius
    # 2-16 cells; 2.6 -> 1.0 degrees at radius 2-4).  On planes and on
    # radius 16-32 MYC stays ahead (its centred columns are exact for
    # unsaturated planes), and the judged estimator keeps MYC there.
    assert all(c > 1000 for c in rep["bin_count"])
    for b in (1, 2, 3):
        assert rep["bin_mean_deg_mlp"][b] < rep["bin_mean_deg_myc"][b], b
    assert rep["bin_mean_deg_combined"][0] <= rep["bin_mean_deg_myc"][0] + 0.05


@pytest.mark.parametrize("radius", [4.0, 8.0])
def test_translated_sphere_shape_error(vof, radius):
    """A sphere carried by a uniform oblique velocity for 16 cells along z:
    L1 distance to the exact translated sphere with the trained network
    (MYC fallback) and with MYC alone, same FP32 step otherwise."""
    from paper_2407_07463_gb300 import synth
    tp = vof.train_params(n_train=4_000_000, n_test=10_000, epochs=4, batch=16384, seed=7)
    wts, _ = vof.vof_mlp_train(tp, DEV)
    shape = (48, 40, 40)
    c0 = np.array([[15.3, 16.7, 12.4]])
    vel = np.array([0.3, 0.2, 1.0])
    u = synth.uniform_velocity(shape, vel)
    dt, steps = 0.25, 64
    c = synth.sphere_cell_fractions(shape, c0, radius)[None]
    exact = synth.sphere_cell_fractions(shape, c0 + vel * dt * steps, radius)
    errs = {}
    for prec in (1, 2):
        cfg = vof.make_config(shape[2], shape[1], shape[0], k_capacity=1, k_active=1, precision=prec,
                              tag_tau=0.0)
        c_d = torch.from_numpy(c).to(DEV, torch.float32).contiguous()
        u_d = torch.from_numpy(u).to(DEV, torch.float32).contiguous()
        ctx = vof.Context(cfg, c_d, u_d)
        if prec == 2:
            ctx.vof_set_mlp(wts, 1e-3)
        rep = ctx.vof_step(dt, steps)
        torch.cuda.synchronize()
        errs[prec] = float(np.abs(c_d.cpu().numpy()[0].astype(np.float64) - exact).sum())
        if prec == 2:
            errs["share"] = rep["faces_network"] / max(1, rep["faces_network"] + rep["faces_myc"])
        ctx.close()
    print("radius", radius, "L1 MYC", errs[1], "L1 learned", errs[2], "network share", errs["share"])
    assert errs[2] <= 1.1 * errs[1]
