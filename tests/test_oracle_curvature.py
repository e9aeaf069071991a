"""Pins of the oracle's height-function curvature and surface-tension source
(Section 2.3: f = sum_i gamma kappa_i grad C_i, one curvature per tracer)
against what geometry fixes (no GPU)."""
import numpy as np
import pytest

from paper_2407_07463_gb300 import synth


def surface_fractions(shape, f, n_sub=8):
    """Fractions of the phase below z = f(x, y): in every cell the mean over
    n_sub^2 footprint points of clamp(f - k, 0, 1) -- so a column's sum is
    the same midpoint rule applied to f itself."""
    nz, ny, nx = shape
    s = (np.arange(n_sub) + 0.5) / n_sub
    xs = (np.arange(nx)[:, None] + s[None, :]).ravel()
    ys = (np.arange(ny)[:, None] + s[None, :]).ravel()
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    F = f(X, Y)
    c = np.zeros(shape)
    for k in range(nz):
        c[k] = np.clip(F - k, 0.0, 1.0).reshape(ny, n_sub, nx, n_sub).mean(axis=(1, 3))
    return c


def analytic_kappa(fx, fy, fxx, fyy, fxy):
    g2 = 1.0 + fx * fx + fy * fy
    return -(fxx * (1 + fy * fy) + fyy * (1 + fx * fx) - 2 * fxy * fx * fy) / g2 ** 1.5


def test_plane_has_zero_curvature(oracle):
    """The column sums of a plane are exactly linear across columns: every
    defined curvature is 0 to rounding, and most interfacial cells have one."""
    rng = np.random.default_rng(3)
    for _ in range(4):
        sx, sy = rng.uniform(-0.6, 0.6, 2)
        c = surface_fractions((20, 18, 18), lambda x, y: 9.3 + sx * (x - 9) + sy * (y - 9))
        kap = oracle.curvature(c)
        inner = np.zeros(c.shape, bool)
        inner[:, 4:-4, 4:-4] = True  # away from the (non-periodic) plane's seams
        interf = (c > 0) & (c < 1) & inner
        ok = interf & np.isfinite(kap)
        assert ok.sum() >= 0.9 * interf.sum() > 0
        assert np.abs(kap[ok]).max() <= 1e-12


@pytest.mark.parametrize("flip", [False, True])
def test_quadratic_surface_exact(oracle, flip):
    """z = f(x, y) quadratic: a column's height is f's footprint mean, which
    differs from f at the footprint centre by the same constant in every
    column, so the centred differences are f's exact derivatives there and
    the discrete curvature equals the surface's curvature at the column
    centre.  The complementary field (phase above) has the opposite sign."""
    a, b, e = 0.05, 0.03, 0.02

    def f(x, y):
        X, Y = x - 8.1, y - 7.7
        return 10.3 + a * X * X + b * Y * Y + e * X * Y

    c = surface_fractions((24, 16, 16), f)
    if flip:
        c = 1.0 - c
    kap = oracle.curvature(c)
    nz, ny, nx = c.shape
    checked = 0
    for k in range(nz):
        for j in range(4, ny - 4):
            for i in range(4, nx - 4):
                if not (0 < c[k, j, i] < 1) or not np.isfinite(kap[k, j, i]):
                    continue
                X, Y = i + 0.5 - 8.1, j + 0.5 - 7.7
                want = analytic_kappa(2 * a * X + e * Y, 2 * b * Y + e * X, 2 * a, 2 * b, e)
                assert kap[k, j, i] == pytest.approx(-want if flip else want, abs=1e-10)
                checked += 1
    assert checked >= 40


def test_sphere_curvature_converges(oracle):
    """Spheres of radius R: the mean curvature over the cells that have one
    is 2/R within 2% at R = 6 and the error shrinks at R = 12; the
    complementary field (a bubble in the phase) gives -2/R."""
    errs = []
    for R in (6.0, 12.0):
        n = int(2 * R + 10)
        cen = np.array([[n / 2 + 0.31, n / 2 - 0.27, n / 2 + 0.13]])
        c = synth.sphere_cell_fractions((n, n, n), cen, R)
        kap = oracle.curvature(c)
        ok = np.isfinite(kap)
        assert ok.sum() >= 0.8 * ((c > 0) & (c < 1)).sum()
        errs.append(abs(kap[ok].mean() * R / 2 - 1))
        kb = oracle.curvature(1.0 - c)
        assert kb[np.isfinite(kb)].mean() == pytest.approx(-2 / R, rel=0.03)
    assert errs[0] < 0.02 and errs[1] < errs[0]


def test_surface_tension_force_on_half_a_drop(oracle):
    """Summed over the z-faces above a sphere's equator, f_z h^3 telescopes
    along each column to -gamma kappa C(equator) h^2, i.e. the force
    -gamma (2/R) pi R^2 = -2 pi gamma R on the upper half (Laplace); the
    whole domain sums to about zero, and a second, distant drop in another
    field adds its own force."""
    R, n, gamma = 8.0, 40, 0.7
    cen = np.array([[20.4, 19.7, 20.0]])
    c1 = synth.sphere_cell_fractions((n, n, n), cen, R)
    k1 = oracle.curvature(c1)
    f = oracle.surface_tension(c1, k1, gamma)
    up = f[2][21:].sum()  # low z-faces of the cells above the equator plane z = 20
    assert up == pytest.approx(-2 * np.pi * gamma * R, rel=0.03)
    assert abs(f[2].sum()) <= 0.02 * abs(up)
    assert np.abs(oracle.surface_tension(c1, np.zeros_like(c1), gamma)).max() == 0.0
    c2 = np.roll(c1, 20, axis=2)
    k2 = oracle.curvature(c2)
    both = oracle.surface_tension(np.stack([c1, c2]), np.stack([k1, k2]), gamma)
    np.testing.assert_allclose(both, f + oracle.surface_tension(c2, k2, gamma), atol=1e-14)
