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
