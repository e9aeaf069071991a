"""Pins of the oracle's learned-normal pieces: backprop against finite
differences, and the canonical frame's invariance (no GPU)."""
import numpy as np
import pytest


def test_backprop_matches_finite_differences(oracle):
    O = oracle
    rng = np.random.default_rng(0)
    p = rng.normal(size=O.MLP_NPARAM) * 0.2
    x = rng.normal(size=(6, 27))
    t = rng.normal(size=(6, 3))
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    loss, g = O.mlp_loss_grad(p, x, t, bf16=False)
    live = np.nonzero(g)[0]
    for i in rng.choice(live, 40, replace=False):
        e = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (O.mlp_loss_grad(pp, x, t, False)[0] - O.mlp_loss_grad(pm, x, t, False)[0]) / (2 * e)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_bf16_forward_close_to_fp64(oracle):
    rng = np.random.default_rng(1)
    p = rng.normal(size=oracle.MLP_NPARAM) * 0.2
    for _ in range(20):
        x = rng.uniform(-0.5, 0.5, 27)
        a = oracle.mlp_forward(p, x, bf16=False)
        b = oracle.mlp_forward(p, x, bf16=True)
        assert np.abs(a - b).max() <= 0.05 * (np.abs(a).max() + 0.1)


def test_canonical_frame_invariance(oracle):
    """Reflecting or permuting the stencil leaves the canonical input
    unchanged, and the canonical Youngs components are >= 0 and sorted."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        st = rng.random((3, 3, 3))
        x, sg, pm = oracle.mlp_canon(st)
        y = oracle.youngs(x.reshape(3, 3, 3) + 0.5)
        assert np.all(y >= -1e-15) and y[0] <= y[1] + 1e-15 <= y[2] + 2e-15
        ax = tuple(rng.permutation(3))
        st2 = np.transpose(st, ax)
        for a in range(3):
            if rng.random() < 0.5:
                st2 = np.flip(st2, axis=a)
        x2, _, _ = oracle.mlp_canon(np.ascontiguousarray(st2))
        np.testing.assert_allclose(x2, x, atol=1e-15)


def test_youngs_network_reproduces_youngs(oracle):
    """A network whose weights encode the Youngs stencil gives, through the
    canonical frame and back, the oracle's Youngs normal: pins the frame
    mapping, the layer order and the BF16 pair inputs."""
    from helpers import youngs_network
    p = youngs_network()
    rng = np.random.default_rng(5)
    for _ in range(40):
        st = rng.random((3, 3, 3))
        m, which, amb = oracle.learned_normal(p, st, tol=np.inf)
        assert which == 0 and amb == 0
        np.testing.assert_allclose(m, oracle.youngs(st), atol=2e-5)


def test_residual_axis_plane_by_hand(oracle):
    """Normal (0,0,1): the plane through the centre cell with fraction c0
    fills the layer below, cuts the middle layer at c0 and leaves the layer
    above empty, so the residual is the mean of |1 - c|, |c0 - c|, |0 - c|
    over the three layers."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        st = rng.random((3, 3, 3))
        c0 = st[1, 1, 1]
        want = (np.abs(1.0 - st[0]).sum() + np.abs(c0 - st[1]).sum() + np.abs(st[2]).sum()) / 27
        assert oracle.normal_residual(st, [0.0, 0.0, 1.0]) == pytest.approx(want, abs=1e-13)
        # the opposite normal swaps the full and empty layers
        want2 = (np.abs(st[0]).sum() + np.abs(c0 - st[1]).sum() + np.abs(1.0 - st[2]).sum()) / 27
        assert oracle.normal_residual(st, [0.0, 0.0, -2.0]) == pytest.approx(want2, abs=1e-13)


def test_residual_zero_on_exact_plane(oracle):
    from helpers import plane_stencil
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.abs(n).sum()
        st = plane_stencil(oracle, n, rng.uniform(-0.2, 0.2))
        assert oracle.normal_residual(st, n) < 1e-13
        assert oracle.normal_residual(st, n + rng.normal(scale=0.2, size=3)) > 1e-4


def test_fallback_decisions(oracle):
    """Exact plane with unsaturated columns: MYC is exact and Youngs is not,
    so the Youngs network falls back to MYC unless the tolerance admits it;
    an all-zero network always falls back; ambiguity follows amb_eps."""
    from helpers import plane_stencil, youngs_network
    p = youngs_network()
    n = np.array([0.15, -0.25, 0.6])
    n /= np.abs(n).sum()
    st = plane_stencil(oracle, n, 0.05)
    e_y = oracle.normal_residual(st, oracle.youngs(st))
    assert e_y > 1e-4 and oracle.normal_residual(st, oracle.myc(st)) < 1e-13
    m, which, _ = oracle.learned_normal(p, st, tol=0.0)
    assert which == 1
    np.testing.assert_allclose(m, n, atol=1e-14)
    m, which, _ = oracle.learned_normal(p, st, tol=2 * e_y)
    assert which == 0
    _, which, amb = oracle.learned_normal(p, st, tol=e_y, amb_eps=1e-3, amb_choice=1)
    assert amb == 1 and which == 1
    _, which, amb = oracle.learned_normal(np.zeros(7312), st, tol=1e9)
    assert which == 1 and amb == 0


def test_learned_step_with_null_network_is_the_myc_step(oracle):
    """A network with all-zero weights has no finite normal: every donor
    falls back to MYC and the step equals the plain step bit for bit."""
    from paper_2407_07463_gb300 import synth
    w = synth.config_small()
    a, ca = oracle.advect_step(w.c, w.u, w.dt, 1.0, 1)
    b, cb, counts = oracle.advect_step_learned(w.c, w.u, w.dt, 1.0, 1, np.zeros(7312))
    assert np.array_equal(a, b) and np.array_equal(ca, cb)
    assert counts[0] == 0 and counts[1] > 0 and counts[2] == 0


def _bf16(a):
    """Round to the nearest BF16 (ties to even) through FP32 (numpy)."""
    f = np.asarray(a, dtype=np.float32).copy()
    b = f.view(np.uint32)
    b += np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))
    b &= np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


def _fwd_layers(p, x):
    """FP64 forward with BF16 weights: layer inputs |x|, |h1|, |h2| and the
    absolute weights, for the error bound below."""
    W1 = _bf16(p[0:2048].reshape(64, 32)[:, :27])
    W2 = _bf16(p[2048:6144].reshape(64, 64))
    W3 = _bf16(p[6144:7168].reshape(16, 64)[:3])
    b1, b2 = p[7168:7232], p[7232:7296]
    h1 = np.maximum(W1 @ x + b1, 0.0)
    h2 = np.maximum(W2 @ h1 + b2, 0.0)
    return (W1, W2, W3), (np.abs(x), h1, h2)


def test_pair_inputs_within_their_error_bound_of_fp64_inputs(oracle):
    """The (hi, lo) BF16 pair the oracle feeds to every layer carries its
    value v to within eps |v|, eps = 2^-17: |v - hi| <= 2^-9 |v| (hi = bf16(v)),
    fl32(v) - hi is exact and lo = bf16 of it adds at most 2^-9 of that,
    plus 2^-24 |v| from the FP32 conversion.  Propagated through the layers
    (ReLU is 1-Lipschitz): d1 = |W1| eps|x|, e1 = d1 + eps|h1|,
    e2 = |W2| e1 + eps|h2|, |d out| <= |W3| e2 (to first order).  The
    pair-input forward (the tensor cores' arithmetic) must lie within that
    bound of the forward on exact FP64 inputs with the same BF16 weights (the
    survey's reading).  A forward that dropped the low halves departs from
    the FP64-input forward by more than 20 times as much in every trial, so
    a wrong split would not hide inside the comparison."""
    rng = np.random.default_rng(11)
    eps = 2.0 ** -17
    worst = 0.0
    for trial in range(60):
        p = rng.normal(size=oracle.MLP_NPARAM) * (0.2 if trial % 2 else 0.5)
        x = rng.uniform(-0.5, 0.5, 27)
        pair = oracle.mlp_forward(p, x, bf16=True)
        exact = oracle.mlp_forward(p, x, bf16="weights")
        (W1, W2, W3), (ax, h1, h2) = _fwd_layers(p, x)
        e1 = np.abs(W1) @ (eps * ax) + eps * h1
        e2 = np.abs(W2) @ e1 + eps * h2
        bound = 1.01 * (np.abs(W3) @ e2) + 1e-15
        assert np.all(np.abs(pair - exact) <= bound), (trial, pair - exact, bound)
        worst = max(worst, float((np.abs(pair - exact) / bound).max()))
        # hi parts only: errors of 2^-9 |v| per input, far above the bound
        hx = _bf16(x)
        g1 = _bf16(np.maximum(W1 @ hx + p[7168:7232], 0.0))
        g2 = _bf16(np.maximum(W2 @ g1 + p[7232:7296], 0.0))
        hi_only = W3 @ g2 + p[7296:7299]
        assert np.abs(hi_only - exact).max() > 20 * np.abs(pair - exact).max(), trial
    print("largest share of the bound used by the pair forward:", worst)


def test_ambiguity_map_marks_both_cells_of_a_face(oracle):
    """With every decision ambiguous, each face whose two branches give
    different fluxes marks both cells it separates, whichever way the
    velocity points: along x, under a uniform velocity of either sign, no
    marked cell is without a marked neighbour along x."""
    from helpers import youngs_network
    from paper_2407_07463_gb300 import synth
    shape = (12, 14, 16)
    c = synth.sphere_cell_fractions(shape, np.array([[8.3, 7.1, 6.2]]), 4.0)[None]
    p = youngs_network(0.05, seed=4)
    for sgn in (1.0, -1.0):
        u = np.zeros((3,) + shape)
        u[0] = 0.8 * sgn
        amb = np.zeros(c.shape, dtype=np.uint8)
        oracle.advect_step_learned(c, u, 0.25, 1.0, 0, p, tol=0.0, amb_eps=1e9, amb_map=amb)
        m = amb[0].astype(bool)
        assert m.sum() > 20
        paired = m & (np.roll(m, 1, axis=2) | np.roll(m, -1, axis=2))
        assert np.array_equal(paired, m), sgn
