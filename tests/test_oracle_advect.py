"""Pins of the oracle's split advection step: exact volume conservation,
exact translation of a plane and of a sphere at CFL 1 (no GPU)."""
import numpy as np
import pytest

from helpers import plane_field
from paper_2407_07463_gb300 import synth


def test_conservation_solenoidal(oracle):
    shape = (20, 24, 28)
    cen = synth.rsa_centres(shape, 4.0, 4, seed=5)
    col, _ = synth.greedy_colours(shape, cen, 4.0, 2)
    c = synth.coloured_fields(shape, cen, 4.0, col, int(col.max()) + 1)
    u = synth.solenoidal_velocity(shape, 6, 0.5, 1.0, seed=6)
    dt = synth.dt_for_cfl(u, 0.3)
    for step in range(3):
        c1, clipped = oracle.advect_step(c, u, dt, 1.0, step)
        for f in range(c.shape[0]):
            before = c[f].sum()
            assert abs(c1[f].sum() + clipped[f] - before) <= 1e-13 * before
            assert abs(clipped[f]) <= 1e-12 * before
        assert c1.min() >= 0.0 and c1.max() <= 1.0
        c = c1


def test_constant_fields_stay(oracle):
    shape = (8, 8, 8)
    u = synth.solenoidal_velocity(shape, 4, 0.4, 0.0, seed=9)
    dt = synth.dt_for_cfl(u, 0.4)
    c = np.stack([np.zeros(shape), np.ones(shape)])
    c1, _ = oracle.advect_step(c, u, dt, 1.0, 0)
    assert np.all(c1[0] == 0.0)
    assert np.abs(c1[1] - 1.0).max() <= 1e-15


def test_plane_translation(oracle):
    """A plane moved by a uniform u = (0,0,1) at CFL 1/4 for 4 steps is the
    initial field rolled by one cell (away from the x/y seams of the
    non-periodic plane)."""
    shape = (16, 10, 10)
    n = np.array([0.12, -0.08, 1.0])
    n /= np.abs(n).sum()
    c0 = plane_field(oracle, shape, n, (5.0, 5.0, 7.3))
    u = synth.uniform_velocity(shape, (0.0, 0.0, 1.0))
    c = c0.copy()
    for s in range(4):
        c, _ = oracle.advect_step(c, u, 0.25, 1.0, s)
    want = np.roll(c0, 1, axis=0)
    inner = (slice(None), slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(c[inner], want[inner], atol=1e-12, rtol=0)


def test_sphere_cfl_one_is_a_roll(oracle):
    """At |s| = 1 every donor empties entirely into its neighbour, whatever
    its reconstruction: the field moves by exactly one cell."""
    shape = (16, 16, 16)
    c0 = synth.sphere_cell_fractions(shape, [(7.3, 8.1, 7.7)], 4.2)
    for d, vec in enumerate(((1.0, 0, 0), (0, 1.0, 0), (0, 0, -1.0))):
        u = synth.uniform_velocity(shape, vec)
        c, _ = oracle.advect_step(c0, u, 1.0, 1.0, 0)
        axis = 2 - d
        shift = -1 if vec[d] < 0 else 1
        np.testing.assert_allclose(c, np.roll(c0, shift, axis=axis), atol=1e-15, rtol=0)


def test_sweep_order_rotates(oracle):
    shape = (12, 12, 12)
    c0 = synth.sphere_cell_fractions(shape, [(6.2, 5.9, 6.1)], 3.3)
    u = synth.solenoidal_velocity(shape, 4, 0.5, 0.3, seed=3)
    dt = synth.dt_for_cfl(u, 0.3)
    a, _ = oracle.advect_step(c0, u, dt, 1.0, 0)
    b, _ = oracle.advect_step(c0, u, dt, 1.0, 3)
    c, _ = oracle.advect_step(c0, u, dt, 1.0, 1)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_openmp_build_equals_serial(oracle):
    """The OpenMP build (z-planes in parallel) gives the serial build's
    step bit for bit, with the same face counts and ambiguity map."""
    if oracle.lib(omp=True) is None:
        pytest.skip("no OpenMP build")
    from helpers import youngs_network
    shape = (18, 20, 22)
    cen = synth.rsa_centres(shape, 4.0, 5, seed=8)
    col, _ = synth.greedy_colours(shape, cen, 4.0, 2)
    c = synth.coloured_fields(shape, cen, 4.0, col, int(col.max()) + 1)
    u = synth.solenoidal_velocity(shape, 6, 0.5, 1.0, seed=9)
    dt = synth.dt_for_cfl(u, 0.3)
    a, ca = oracle.advect_step(c, u, dt, 1.0, 2)
    b, cb = oracle.advect_step(c, u, dt, 1.0, 2, omp=True)
    assert np.array_equal(a, b) and np.array_equal(ca, cb)
    p = youngs_network(0.02, seed=3)
    ma = np.zeros(c.shape, dtype=np.uint8)
    mb = np.zeros(c.shape, dtype=np.uint8)
    a, ca, na = oracle.advect_step_learned(c, u, dt, 1.0, 1, p, amb_eps=3e-5, amb_map=ma)
    b, cb, nb = oracle.advect_step_learned(c, u, dt, 1.0, 1, p, amb_eps=3e-5, amb_map=mb, omp=True)
    assert np.array_equal(a, b) and np.array_equal(ca, cb) and na == nb
    assert np.array_equal(ma, mb)
    assert na[0] > 0 and na[1] > 0
