"""Pins of the oracle's drop table and nearest-particle statistics (Section 3,
Section 4.3-4.4) against closed forms and the values the paper prints."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from paper_2407_07463_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def lattice_field(n_per_axis, spacing, radius):
    L = n_per_axis * spacing
    shape = (L, L, L)
    g = (np.arange(n_per_axis) + 0.5) * spacing
    cen = np.array([(x, y, z) for z in g for y in g for x in g])
    return shape, cen, synth.sphere_cell_fractions(shape, cen, radius)


def test_drop_table_lattice(oracle):
    """Spheres centred on a lattice of cell centres: volumes equal, centroids
    exact by symmetry (including drops cut by the periodic boundary)."""
    shape, cen, c = lattice_field(3, 10, 3.2)
    c = np.roll(c, (5, 3, 7), axis=(0, 1, 2))  # drops straddle the wrap
    lab, n = oracle.label(c)
    assert n == 27
    vol, got = oracle.drop_table(c, lab, n)
    want = (cen + np.array([7, 3, 5])) % 30
    for p in got:
        dlt = want - p
        dlt -= 30 * np.round(dlt / 30)
        assert np.abs(dlt).max(axis=1).min() <= 1e-12
    assert np.all((got >= 0) & (got < 30))
    np.testing.assert_allclose(vol, vol[0], rtol=1e-14)


def test_lattice_statistics(oracle):
    """Cubic lattice: 6 equidistant nearest neighbours (h = 1/6), M = 0,
    A = 0, tr R = spacing^2 (Section 3 definitions)."""
    shape, cen, c = lattice_field(4, 12, 3.0)
    lab, n = oracle.label(c)
    vol, got = oracle.drop_table(c, lab, n)
    d = (6 * vol.mean() / math.pi) ** (1 / 3)
    ps = oracle.PairStats(n_rbins=200, dr=d / 100).add(got, [48.0] * 3, tie_tol=1e-12 * d)
    assert ps.E == n
    np.testing.assert_allclose(ps.M, 0.0, atol=1e-10)
    np.testing.assert_allclose(ps.A, 0.0, atol=1e-9)
    assert np.trace(ps.R) == pytest.approx(144.0, rel=1e-12)
    k = int(math.floor(12.0 / (d / 100)))
    assert ps.hist_r[k] == pytest.approx(n, rel=1e-12)
    # theta histogram: 1/6 of the weight at theta = 0, 1/6 at pi, 4/6 at pi/2
    hrt = ps.hist_rt.reshape(-1, 150)[k]
    assert hrt[0] == pytest.approx(n / 6) and hrt[149] == pytest.approx(n / 6)
    assert hrt[75] == pytest.approx(4 * n / 6)


def test_lattice_distance_printed_value(oracle):
    """Section 4.3 prints the cubic-lattice nearest distance
    1/2 [4 pi / (3 phi)]^(1/3) ~ 3.74 d at phi = 0.01; the statistics of a
    lattice of drops at phi = 0.01 must give that distance."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["lattice_nearest_over_d"]
    phi = gold["phi"]
    d = 2.0  # diameter in cells of point drops; only centroids enter here
    a = d * (math.pi / (6 * phi)) ** (1 / 3)
    g = (np.arange(4) + 0.5) * a
    cen = np.array([(x, y, z) for z in g for y in g for x in g])
    ps = oracle.PairStats(n_rbins=1000, dr=d / 100).add(cen, [4 * a] * 3, tie_tol=1e-12 * d)
    r = math.sqrt(np.trace(ps.R))
    assert r / d == pytest.approx(gold["value"], abs=gold["abs_tol"])
    assert r / d == pytest.approx(0.5 * (4 * math.pi / (3 * phi)) ** (1 / 3), rel=1e-12)


def test_two_drop_moments(oracle):
    cen = np.array([[10.0, 10.0, 10.0], [13.0, 14.0, 10.0]])
    ps = oracle.PairStats(n_rbins=100, dr=0.1).add(cen, [40.0] * 3)
    r = np.array([3.0, 4.0, 0.0])
    assert ps.E == 2
    np.testing.assert_allclose(ps.M, 0.0, atol=1e-15)
    np.testing.assert_allclose(ps.R, np.outer(r, r), atol=1e-13)
    assert ps.hist_r[50] == 2.0  # |r| = 5 -> bin 50 of width 0.1
    # theta from the vertical (z) axis is pi/2 for both events
    assert ps.hist_rt.reshape(-1, 150)[50][75] == 2.0


def test_minimum_image(oracle):
    cen = np.array([[0.5, 5.0, 5.0], [19.5, 5.0, 5.0], [10.0, 5.0, 5.0]])
    ps = oracle.PairStats(n_rbins=100, dr=0.5).add(cen, [20.0, 20.0, 20.0])
    # drops 0 and 1 are 1 apart through the x wrap
    assert ps.hist_r[2] == 2.0


def test_poisson_points_mean_square_distance(oracle):
    """Poisson points: P(r) = 4 pi r^2 n exp(-4/3 pi n r^3), hence
    <r^2> = Gamma(5/3) (4 pi n / 3)^(-2/3)."""
    rng = np.random.default_rng(51)
    L = 60.0
    n = 4000
    cen = rng.random((n, 3)) * L
    ps = oracle.PairStats(n_rbins=100, dr=0.1).add(cen, [L] * 3)
    dens = n / L ** 3
    want = special.gamma(5 / 3) * (4 * math.pi * dens / 3) ** (-2 / 3)
    assert np.trace(ps.R) == pytest.approx(want, rel=0.04)
    np.testing.assert_allclose(ps.M, 0.0, atol=0.05 * math.sqrt(want))
    assert np.abs(ps.A).max() < 0.06 * want


def dilute(r, d, phi):
    n_p = 6 * phi / (math.pi * d ** 3)
    return n_p * math.exp(-8 * phi * ((r / d) ** 3 - 1))


@pytest.mark.parametrize("phi", [0.01, 0.05, 0.1, 0.2])
def test_dilute_closed_forms(phi):
    """Section 4.3 eq. Pnst_dilute integrates to 1 over r >= d, and its second
    moment is the closed form of Section 4.4 for r_m^2."""
    d = 1.0
    norm = integrate.quad(lambda r: 4 * math.pi * r * r * dilute(r, d, phi), d, np.inf)[0]
    assert norm == pytest.approx(1.0, abs=1e-10)
    m2 = integrate.quad(lambda r: 4 * math.pi * r ** 4 * dilute(r, d, phi), d, np.inf)[0]
    closed = special.gammaincc(5 / 3, 8 * phi) * special.gamma(5 / 3) / 8 ** (2 / 3) \
        * math.exp(8 * phi) / phi ** (2 / 3)
    assert m2 == pytest.approx(closed, rel=1e-10)


def test_torquato_reduces_to_dilute():
    """Section 4.3 eq. torquato: e -> 1, f, g -> 0 as phi -> 0."""
    for r in (1.0, 1.5, 3.0):
        phi = 1e-7
        e = (1 + phi) / (1 - phi) ** 3
        f = -phi * (3 + phi) / (2 * (1 - phi) ** 3)
        g = phi ** 2 / (2 * (1 - phi) ** 3)
        n_p = 6 * phi / math.pi
        th = n_p * (e + f / r + g / r ** 2) * math.exp(
            -phi * (8 * e * (r ** 3 - 1) + 12 * f * (r ** 2 - 1) + 24 * g * (r - 1)))
        assert th == pytest.approx(dilute(r, 1.0, phi), rel=1e-6)


def test_rsa_dilute_agrees_with_closed_form(oracle):
    """Hard spheres placed at random at phi = 0.01 follow eq. Pnst_dilute to
    O(phi): tr R / r_m^2 ~ 1 (Section 4.4 compares DNS with r_m this way)."""
    phi = 0.01
    d = 2.0
    L = 100.0
    n = int(round(phi * L ** 3 / (math.pi / 6 * d ** 3)))
    shape = (int(L),) * 3
    vals = []
    for seed in range(3):
        cen = synth.rsa_centres(shape, d / 2, n, 300 + seed)
        ps = oracle.PairStats(n_rbins=100, dr=d / 100).add(cen, [L] * 3)
        vals.append(np.trace(ps.R))
    rm2 = special.gammaincc(5 / 3, 8 * phi) * special.gamma(5 / 3) / 8 ** (2 / 3) \
        * math.exp(8 * phi) / phi ** (2 / 3) * d * d
    assert np.mean(vals) / rm2 == pytest.approx(1.0, abs=0.05)


# ---------------------------------------------------------------- drop shape (Appendix A)


def ellipsoid_fractions(shape, centre, axes, rot_z=0.0, n_sub=6):
    """Cell fractions of an ellipsoid (semi-axes `axes` along x, y, z after a
    rotation by rot_z about z), by n_sub^3 midpoint samples per cell."""
    nz, ny, nx = shape
    s = (np.arange(n_sub) + 0.5) / n_sub
    ca, sa = np.cos(rot_z), np.sin(rot_z)
    out = np.zeros(shape)
    zs = (np.arange(nz)[:, None] + s[None, :]).ravel()
    ys = (np.arange(ny)[:, None] + s[None, :]).ravel()
    xs = (np.arange(nx)[:, None] + s[None, :]).ravel()
    Z, Y, X = np.meshgrid(zs - centre[2], ys - centre[1], xs - centre[0], indexing="ij")
    u = ca * X + sa * Y
    v = -sa * X + ca * Y
    inside = (u / axes[0]) ** 2 + (v / axes[1]) ** 2 + (Z / axes[2]) ** 2 < 1.0
    return inside.reshape(nz, n_sub, ny, n_sub, nx, n_sub).mean(axis=(1, 3, 5))


def test_inertia_of_one_and_two_full_cells_by_hand(oracle):
    """One full cell: I = h^5/6 delta (the cube's own moment), chi = 1.  Two
    full cells side by side along x: r = +-h/2 x, so I_xx = h^5/3 and
    I_yy = I_zz = 2 h^3 (h/2)^2 + h^5/3 = 5 h^5/6, chi = sqrt(5/2)."""
    for h in (1.0, 2.0):
        c = np.zeros((6, 6, 6))
        lab = np.zeros(c.shape, dtype=np.int32)
        c[2, 3, 1] = 1.0
        lab[2, 3, 1] = 1
        I, chi = oracle.drop_inertia(c, lab, 1, h=h)
        np.testing.assert_allclose(I[0], np.array([1, 1, 1, 0, 0, 0]) * h ** 5 / 6, rtol=1e-14, atol=1e-14)
        assert chi[0] == pytest.approx(1.0, abs=1e-14)
        c[2, 3, 2] = 1.0
        lab[2, 3, 2] = 1
        I, chi = oracle.drop_inertia(c, lab, 1, h=h)
        np.testing.assert_allclose(I[0], np.array([1 / 3, 5 / 6, 5 / 6, 0, 0, 0]) * h ** 5, rtol=1e-14,
                                   atol=1e-14)
        assert chi[0] == pytest.approx(np.sqrt(2.5), rel=1e-14)


def brute_inertia(c, lab, cen, h=1.0):
    """Inertia tensor of the drop's colour density (each cell of the drop
    holding c uniformly) by 2-point Gauss-Legendre quadrature per axis in
    every cell (exact for the quadratic integrand), minimum image."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    nz, ny, nx = c.shape
    L = np.array([nx, ny, nz]) * h
    T = np.zeros((3, 3))
    for k, j, i in zip(*np.nonzero(lab)):
        for gz in g:
            for gy in g:
                for gx in g:
                    r = (np.array([i + gx, j + gy, k + gz]) * h - cen) % L
                    r = np.where(r > 0.5 * L, r - L, r)
                    T += c[k, j, i] * h ** 3 / 8 * (r @ r * np.eye(3) - np.outer(r, r))
    return T


def tensor(I):
    return np.array([[I[0], I[3], I[4]], [I[3], I[1], I[5]], [I[4], I[5], I[2]]])


@pytest.mark.parametrize("rot", [0.0, 0.5])
def test_inertia_of_the_colour_density_by_quadrature(oracle, rot):
    """The tensor of a drop's colour density equals brute-force quadrature
    of it, and the oracle's chi is the square root of the ratio of the
    extreme eigenvalues of its own tensor (an independent eigen-solver)."""
    c = ellipsoid_fractions((14, 20, 24), (12.3, 9.8, 7.2), (7.0, 5.0, 3.5), rot)
    lab = (c > 0).astype(np.int32)
    _, cen = oracle.drop_table(c, lab, 1, h=0.5)
    I, chi = oracle.drop_inertia(c, lab, 1, h=0.5)
    np.testing.assert_allclose(tensor(I[0]), brute_inertia(c, lab, cen[0], h=0.5), rtol=1e-12, atol=1e-12)
    ev = np.linalg.eigvalsh(tensor(I[0]))
    assert chi[0] == pytest.approx(np.sqrt(ev[-1] / ev[0]), rel=1e-12)


def test_inertia_converges_to_the_sharp_ellipsoid(oracle):
    """Against the sharp ellipsoid of semi-axes (a, b, c) -- principal moments
    V(b^2+c^2)/5, V(a^2+c^2)/5, V(a^2+b^2)/5 -- the colour density's moments
    err by O(h / size) (the fluid of a cut cell is spread over the cell):
    within 3% at axes (10, 7, 5) cells, and at most 0.6 of that when the
    ellipsoid is twice as large; chi within 1% and 0.5%."""
    errs, cerrs = [], []
    for s in (1, 2):
        a, b, cz = 10.0 * s, 7.0 * s, 5.0 * s
        # the box is more than twice the drop (minimum image about the centroid)
        c = ellipsoid_fractions((22 * s + 2, 32 * s, 42 * s + 2), (21.3 * s, 15.8 * s, 11.2 * s + 1),
                                (a, b, cz), 0.4, n_sub=4)
        lab = (c > 0).astype(np.int32)
        I, chi = oracle.drop_inertia(c, lab, 1)
        V = 4.0 / 3.0 * np.pi * a * b * cz
        want = np.sort([V * (b * b + cz * cz) / 5, V * (a * a + cz * cz) / 5, V * (a * a + b * b) / 5])
        ev = np.linalg.eigvalsh(tensor(I[0]))
        errs.append(np.abs(ev / want - 1).max())
        cerrs.append(abs(chi[0] / np.sqrt(want[-1] / want[0]) - 1))
    print("relative moment errors", errs, "chi errors", cerrs)
    assert errs[0] < 0.03 and errs[1] < 0.6 * errs[0]
    assert cerrs[0] < 0.01 and cerrs[1] < 0.005


def test_inertia_across_the_periodic_boundary(oracle):
    """The same drop shifted so that it straddles the periodic faces keeps
    its tensor."""
    shape = (24, 28, 32)
    c = ellipsoid_fractions(shape, (16.3, 13.8, 12.2), (8.0, 5.0, 4.0), 0.3)
    lab = (c > 0).astype(np.int32)
    I0, chi0 = oracle.drop_inertia(c, lab, 1)
    c2 = np.roll(c, (11, 13, 17), axis=(0, 1, 2))
    I1, chi1 = oracle.drop_inertia(c2, np.roll(lab, (11, 13, 17), axis=(0, 1, 2)), 1)
    np.testing.assert_allclose(I1, I0, rtol=1e-11, atol=1e-9)
    assert chi1[0] == pytest.approx(chi0[0], rel=1e-11)
