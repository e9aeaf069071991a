"""Pins of the oracle's PLIC geometry and normals against closed forms,
brute-force quadrature and invariants (no GPU)."""
import itertools
import math

import numpy as np
import pytest

from helpers import plane_stencil


def chord_quadrature_volume(m, alpha, n=1200):
    """Volume of {m.x < alpha} in the unit cube by midpoint quadrature over the
    two axes other than the one with the largest |m|, with the analytic extent
    along that axis (independent of the oracle's face-clipping formula)."""
    m = np.asarray(m, dtype=np.float64)
    a = int(np.argmax(np.abs(m)))
    b, c = [t for t in range(3) if t != a]
    g = (np.arange(n) + 0.5) / n
    Y, Z = np.meshgrid(g, g, indexing="ij")
    rest = alpha - m[b] * Y - m[c] * Z
    if m[a] > 0:
        ext = np.clip(rest / m[a], 0.0, 1.0)
    else:
        ext = 1.0 - np.clip(rest / m[a], 0.0, 1.0)
    return float(ext.mean())


def test_volume_closed_forms(oracle):
    O = oracle
    for d in range(3):
        e = np.zeros(3)
        e[d] = 1.0
        for a in (0.0, 0.1, 0.37, 1.0):
            assert O.plic_volume(e, a) == pytest.approx(a, abs=1e-15)
    # corner simplex x+y+z < a (a <= 1): a^3 / 6
    for a in (0.05, 0.3, 0.9, 1.0):
        assert O.plic_volume([1, 1, 1], a) == pytest.approx(a ** 3 / 6, abs=1e-15)
    # triangle prism x+y < a: a^2/2 for a <= 1, 1-(2-a)^2/2 for a >= 1
    for a in (0.2, 0.8, 1.3, 1.9):
        want = a * a / 2 if a <= 1 else 1 - (2 - a) ** 2 / 2
        assert O.plic_volume([1, 1, 0], a) == pytest.approx(want, abs=1e-15)
    assert O.plic_volume([1, 1, 1], 1.5) == pytest.approx(0.5, abs=1e-15)
    assert O.plic_volume([0.3, -0.2, 0.5], -0.2) == 0.0
    assert O.plic_volume([0.3, -0.2, 0.5], 0.8) == pytest.approx(1.0, abs=1e-15)


def test_volume_against_quadrature(oracle):
    rng = np.random.default_rng(11)
    for _ in range(40):
        m = rng.normal(size=3)
        m /= np.abs(m).sum()
        lo = m[m < 0].sum()
        hi = m[m > 0].sum()
        alpha = lo + rng.random() * (hi - lo)
        assert oracle.plic_volume(m, alpha) == pytest.approx(
            chord_quadrature_volume(m, alpha), abs=2e-6)


def test_volume_symmetries(oracle):
    O = oracle
    rng = np.random.default_rng(12)
    for _ in range(200):
        m = rng.normal(size=3)
        alpha = rng.normal()
        v = O.plic_volume(m, alpha)
        # complement
        assert v + O.plic_volume(-m, -alpha) == pytest.approx(1.0, abs=2e-15)
        # reflection x_0 -> 1 - x_0
        mr = m.copy()
        mr[0] = -m[0]
        assert O.plic_volume(mr, alpha - m[0]) == pytest.approx(v, abs=2e-15)
        # axis permutation
        p = rng.permutation(3)
        assert O.plic_volume(m[p], alpha) == pytest.approx(v, abs=2e-15)
        # scale invariance
        assert O.plic_volume(3.0 * m, 3.0 * alpha) == pytest.approx(v, abs=2e-15)


def test_alpha_inverts_volume(oracle):
    """V(m, alpha(m, c)) = c across the cube (10^4 points)."""
    O = oracle
    rng = np.random.default_rng(13)
    worst = 0.0
    for t in range(10000):
        m = rng.normal(size=3)
        if t % 5 == 0:
            m[rng.integers(3)] = 0.0  # degenerate normals
        m /= np.abs(m).sum()
        c = rng.random() if t % 7 else 10.0 ** rng.uniform(-12, -1)
        if t % 2:
            c = 1.0 - c
        a = O.plic_alpha(m, c)
        worst = max(worst, abs(O.plic_volume(m, a) - c))
    assert worst <= 1e-14
    assert O.plic_alpha([0.2, 0.3, -0.5], 0.0) == pytest.approx(-0.5)
    assert O.plic_alpha([0.2, 0.3, -0.5], 1.0) == pytest.approx(0.5)


def vertex_gradient_normal(st):
    """Average of the eight vertex gradients of the 3x3x3 stencil, each by
    finite differences over the 2x2x2 cells around the vertex; m = -grad c."""
    g = np.zeros(3)
    for sx, sy, sz in itertools.product((0, 1), repeat=3):
        blk = st[sz:sz + 2, sy:sy + 2, sx:sx + 2]  # [k][j][i]
        g[0] += (blk[:, :, 1] - blk[:, :, 0]).mean()
        g[1] += (blk[:, 1, :] - blk[:, 0, :]).mean()
        g[2] += (blk[1, :, :] - blk[0, :, :]).mean()
    m = -g
    return m / np.abs(m).sum()


def test_youngs_is_vertex_gradient_average(oracle):
    rng = np.random.default_rng(14)
    for _ in range(100):
        st = rng.random((3, 3, 3))
        np.testing.assert_allclose(oracle.youngs(st), vertex_gradient_normal(st), atol=1e-15)


def test_centred_column_hand_example(oracle):
    # columns along z; heights H(i,j) = 1.5 + 0.2 i - 0.1 j of liquid below
    st = np.zeros((3, 3, 3))
    for j in (-1, 0, 1):
        for i in (-1, 0, 1):
            h = 1.5 + 0.2 * i - 0.1 * j
            for k in range(3):
                st[k, j + 1, i + 1] = min(max(h - k, 0.0), 1.0)
    m = oracle.centred_column(st, 2)
    raw = np.array([-0.2, 0.1, 1.0])
    np.testing.assert_allclose(m, raw / np.abs(raw).sum(), atol=1e-15)


def _unsaturated(st, a):
    s = np.moveaxis(st, 2 - a, 0)
    for p, q in [(1, 1), (0, 1), (2, 1), (1, 0), (1, 2)]:
        col = s[:, p, q]
        if {col[0], col[2]} != {0.0, 1.0}:
            return False
    return True


def test_myc_exact_for_planes(oracle):
    """A plane whose centred columns along its dominant axis do not saturate
    is reconstructed exactly (both candidates it may pick are exact)."""
    rng = np.random.default_rng(15)
    tested = 0
    while tested < 150:
        n = rng.normal(size=3)
        n /= np.abs(n).sum()
        off = rng.uniform(-0.5, 0.5) * np.abs(n).max()
        st = plane_stencil(oracle, n, off)
        if not (0 < st[1, 1, 1] < 1) or not _unsaturated(st, int(np.argmax(np.abs(n)))):
            continue
        np.testing.assert_allclose(oracle.myc(st), n, atol=1e-13)
        tested += 1


def test_myc_symmetry(oracle):
    """Reflecting or permuting the stencil reflects or permutes the normal."""
    rng = np.random.default_rng(16)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.abs(n).sum()
        st = plane_stencil(oracle, n, rng.uniform(-0.3, 0.3))
        st = np.clip(st + 0.02 * rng.normal(size=st.shape), 0, 1)
        m = oracle.myc(st)
        # reflect x (array axis 2)
        mr = oracle.myc(st[:, :, ::-1].copy())
        np.testing.assert_allclose(mr, m * np.array([-1, 1, 1]), atol=1e-14)
        # swap x and y (array axes 2 and 1)
        ms = oracle.myc(np.ascontiguousarray(np.swapaxes(st, 1, 2)))
        np.testing.assert_allclose(ms, m[[1, 0, 2]], atol=1e-14)


def test_myc_degenerate(oracle):
    st = np.zeros((3, 3, 3))
    st[1, 1, 1] = 0.5  # isolated cell: Youngs vanishes, centred column along x
    np.testing.assert_allclose(oracle.myc(st), [1.0, 0.0, 0.0])


def test_face_flux_against_quadrature(oracle):
    """Flux = s * fraction of the swept sub-cell under the plane (brute force
    quadrature over the sub-cell, independent of the sub-cell mapping)."""
    rng = np.random.default_rng(17)
    for _ in range(30):
        m = rng.normal(size=3)
        m /= np.abs(m).sum()
        c = rng.uniform(0.05, 0.95)
        alpha = oracle.plic_alpha(m, c)
        d = int(rng.integers(3))
        s = rng.uniform(-0.5, 0.5)
        x0, x1 = (1 - s, 1.0) if s > 0 else (0.0, -s)
        # quadrature: fraction of {x_d in [x0,x1]} x [0,1]^2 with m.x < alpha
        n = 400
        g = (np.arange(n) + 0.5) / n
        gd = x0 + (x1 - x0) * g
        o = [t for t in range(3) if t != d]
        A, B, D = np.meshgrid(g, g, gd, indexing="ij")
        val = m[o[0]] * A + m[o[1]] * B + m[d] * D
        frac = (val < alpha).mean()
        assert oracle.face_flux(m, alpha, d, s) == pytest.approx(s * frac, abs=3e-3 * abs(s) + 1e-12)


def test_cell_face_flux_empty_full(oracle):
    c = np.zeros((4, 4, 4))
    c[1, 1, 1] = 1.0
    # low z-face of cell (1,1,2): donor (1,1,1) when s > 0
    assert oracle.cell_face_flux(c, 1, 1, 2, 2, 0.3) == 0.3
    assert oracle.cell_face_flux(c, 1, 1, 2, 2, -0.3) == 0.0
    assert oracle.cell_face_flux(c, 1, 1, 1, 2, -0.3) == -0.3
    assert oracle.cell_face_flux(c, 1, 1, 1, 2, 0.0) == 0.0
