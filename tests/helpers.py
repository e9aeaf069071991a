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


# layout of the learned estimator's flat parameter vector (FP32 blob order)
MLP_SPANS = {"W1": (0, 2048), "W2": (2048, 6144), "W3": (6144, 7168), "b1": (7168, 7232),
             "b2": (7232, 7296), "b3": (7296, 7312)}


def youngs_network(noise=0.0, seed=0):
    """Parameters of a 27-64-64-3 ReLU network whose output is the Youngs
    gradient estimate of its (canonical) input stencil: hidden units 2a and
    2a+1 of layer 1 hold relu(+y_a) and relu(-y_a) with
    y_a = sum over the 9 (b, c) of w_b w_c [x(-1 along a) - x(+1 along a)],
    w = (1, 2, 1); layer 2 passes units 0..5 through; layer 3 outputs
    y_a = h[2a] - h[2a+1].  All these weights are exact in BF16.  With
    noise > 0 the remaining units get seeded random weights and the three
    outputs a small random dependence on them, so that every weight of the
    network is exercised while the output stays close to Youngs."""
    p = np.zeros(7312)
    W1 = p[0:2048].reshape(64, 32)
    W2 = p[2048:6144].reshape(64, 64)
    W3 = p[6144:7168].reshape(16, 64)
    b1, b2 = p[7168:7232], p[7232:7296]
    w = (1.0, 2.0, 1.0)
    for a in range(3):
        for u in (-1, 1):
            for b in (-1, 0, 1):
                for cc in (-1, 0, 1):
                    o = [0, 0, 0]
                    o[a] = u
                    o[(a + 1) % 3] = b
                    o[(a + 2) % 3] = cc
                    q = (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1)
                    W1[2 * a, q] = -u * w[b + 1] * w[cc + 1]
                    W1[2 * a + 1, q] = u * w[b + 1] * w[cc + 1]
    for u in range(6):
        W2[u, u] = 1.0
    for a in range(3):
        W3[a, 2 * a] = 1.0
        W3[a, 2 * a + 1] = -1.0
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        W1[6:, :27] = rng.normal(scale=0.3, size=(58, 27))
        b1[6:] = rng.normal(scale=0.1, size=58)
        W2[6:, :] = rng.normal(scale=0.15, size=(58, 64))
        b2[6:] = rng.normal(scale=0.1, size=58)
        W2[:6, 6:] = rng.normal(scale=noise, size=(6, 58))
        W3[:3, 6:] = rng.normal(scale=noise, size=(3, 58))
    return p
