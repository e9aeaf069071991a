"""Small test helpers shared by the oracle and GPU tests (no method arithmetic)."""
import numpy as np


def plane_stencil(O, n, off):
    """3x3x3 stencil st[k][j][i] of the half-space n.x < off (x relative to the
    centre cell's centre), each cell's fraction from the oracle's PLIC volume."""
    st = np.zeros((3, 3, 3))
    for k in (-1, 0, 1):
        for j in (-1, 0, 1):
            for i in (-1, 0, 1):
                alpha = off - (n[0] * (i - 0.5) + n[1] * (j - 0.5) + n[2] * (k - 0.5))
                st[k + 1, j + 1, i + 1] = O.plic_volume(n, alpha)
    return st


def plane_field(O, shape, n, point):
    """Volume fractions of the half-space n.(x - point) < 0 on a grid (cells of
    unit size, cell (i,j,k) = [i,i+1]x[j,j+1]x[k,k+1]); not periodic."""
    nz, ny, nx = shape
    c = np.zeros(shape)
    n = np.asarray(n, dtype=np.float64)
    base = float(n @ np.asarray(point, dtype=np.float64))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c[k, j, i] = O.plic_volume(n, base - (n[0] * i + n[1] * j + n[2] * k))
    return c
