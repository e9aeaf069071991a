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
