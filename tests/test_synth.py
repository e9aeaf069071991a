"""The seeded input generators: determinism and the structural properties the
workloads promise (no method arithmetic here)."""
import numpy as np

from paper_2407_07463_gb300 import synth


def test_rsa_min_distance_and_determinism():
    shape = (40, 40, 40)
    a = synth.rsa_centres(shape, 4.0, 30, seed=7)
    b = synth.rsa_centres(shape, 4.0, 30, seed=7)
    assert np.array_equal(a, b)
    L = np.array([40.0, 40.0, 40.0])
    d = a[:, None, :] - a[None, :, :]
    d -= L * np.round(d / L)
    dist = np.sqrt((d ** 2).sum(-1)) + np.eye(len(a)) * 1e9
    assert dist.min() >= 8.0


def test_velocity_discretely_solenoidal():
    u = synth.solenoidal_velocity((24, 20, 16), 8, 0.5, 1.0, seed=3)
    div = (np.roll(u[0], -1, 2) - u[0]) + (np.roll(u[1], -1, 1) - u[1]) + (np.roll(u[2], -1, 0) - u[2])
    assert np.abs(div).max() < 1e-14
    rand = u.copy()
    rand[2] -= 1.0
    assert abs(np.abs(rand).max() - 0.5) < 1e-12
    assert synth.dt_for_cfl(u, 0.3) * np.abs(u).max() == 0.3


def test_sphere_fractions_volume():
    c = synth.sphere_cell_fractions((24, 24, 24), [(11.3, 12.1, 12.7)], 5.0)
    assert abs(c.sum() - 4 / 3 * np.pi * 125) < 0.1  # quadrature error ~1e-4 relative
    assert c.min() >= 0 and c.max() <= 1


def test_colouring_separates_conflicts():
    shape = (64, 64, 64)
    cen = synth.rsa_centres(shape, 6.0, 60, seed=4)
    col, used = synth.greedy_colours(shape, cen, 6.0, 2)
    dc = synth.conflict_distance(6.0, 2)
    L = 64.0
    for i in range(len(cen)):
        d = cen - cen[i]
        d -= L * np.round(d / L)
        near = (np.sqrt((d ** 2).sum(1)) < dc) & (np.arange(len(cen)) != i)
        assert np.all(col[near] != col[i])
    assert used == col.max() + 1
