"""Seeded synthetic inputs for the multi-field VoF step.

This module builds the *inputs* of the method and nothing else: drop centres
placed by random sequential addition (RSA), cell volume fractions of spheres by
numerical quadrature, a discretely solenoidal face velocity, and a greedy
initial assignment of drops to colour fields.  It holds none of the method's
arithmetic (no PLIC normal, plane constant, flux, labelling or recolouring), so
the FP64 oracle and the CUDA path can both consume what it produces.

The workloads stand in for the paper's direct numerical simulations
(Section 2.1: N_b = 125 mono-disperse drops, d/Delta = 20, phi = 0.01-0.2 in a
tri-periodic cube), whose data is not public: spheres of a fixed radius in cells
at a prescribed volume fraction, advected by a seeded smooth solenoidal field.

Layouts (all C-contiguous, x fastest):
  c[K][nz][ny][nx]   volume fraction of colour field k
  u[3][nz][ny][nx]   u[d] is the velocity on the LOW d-face of the cell
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ---------------------------------------------------------------------------
# drop centres


def rsa_centres(shape, radius, n, seed, min_dist=None, max_attempts=10_000_000):
    """Random sequential addition of ``n`` sphere centres in a periodic box.

    ``shape`` is (nz, ny, nx) in cells (cell size 1); centres are continuous
    positions (x, y, z) in [0, n_axis).  Each new centre is accepted when its
    minimum-image distance to every accepted centre is at least ``min_dist``
    (default 2 * radius, i.e. non-overlapping spheres).
    """
    rng = np.random.default_rng(seed)
    L = np.array([shape[2], shape[1], shape[0]], dtype=np.float64)
    dmin = 2.0 * radius if min_dist is None else float(min_dist)
    nb = np.maximum((L // max(dmin, 1e-9)).astype(int), 1)
    bs = L / nb
    bins: dict = {}
    out = np.empty((n, 3), dtype=np.float64)
    count = 0
    attempts = 0
    while count < n:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError(f"RSA stalled at {count}/{n} spheres")
        p = rng.random(3) * L
        b = (p // bs).astype(int) % nb
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((b[0] + dx) % nb[0], (b[1] + dy) % nb[1], (b[2] + dz) % nb[2])
                    lst = bins.get(key)
                    if not lst:
                        continue
                    q = np.asarray(lst)
                    d = q - p
                    d -= L * np.round(d / L)
                    if np.any(np.einsum("ij,ij->i", d, d) < dmin * dmin):
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[count] = p
            bins.setdefault((b[0], b[1], b[2]), []).append(p)
            count += 1
    return out


def uniform_centres(shape, radius, n, seed):
    """Uniform random non-overlapping centres by rejection (same as RSA)."""
    return rsa_centres(shape, radius, n, seed)


def n_spheres_for_phi(shape, radius, phi):
    """Number of spheres of ``radius`` cells giving volume fraction ``phi``."""
    vol = float(shape[0] * shape[1] * shape[2])
    return int(round(phi * vol / (4.0 / 3.0 * math.pi * radius ** 3)))


# ---------------------------------------------------------------------------
# sphere volume fractions by quadrature


def _gauss_nodes(n_sub, n_gauss):
    x, w = np.polynomial.legendre.leggauss(n_gauss)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    nodes = (np.arange(n_sub)[:, None] + x[None, :]).ravel() / n_sub
    weights = np.tile(w, n_sub) / n_sub
    return nodes, weights


def sphere_cell_fractions(shape, centres, radius, n_sub=2, n_gauss=4, inside=True):
    """Volume fraction of the union of (disjoint) spheres in every cell.

    Cells wholly inside a sphere get 1, cells wholly outside get 0; cut cells
    are integrated with composite Gauss-Legendre quadrature over (x, y) of the
    analytic chord length of the sphere along z.  Returns c[nz][ny][nx].
    With ``inside=False`` the complement (1 - c) is returned.
    """
    nz, ny, nx = shape
    c = np.zeros(shape, dtype=np.float64)
    L = np.array([nx, ny, nz], dtype=np.float64)
    qx, qw = _gauss_nodes(n_sub, n_gauss)
    QX, QY = np.meshgrid(qx, qx, indexing="ij")
    QW = np.outer(qw, qw).ravel()
    QX = QX.ravel()
    QY = QY.ravel()
    r2 = radius * radius
    cut_idx = []
    cut_geo = []
    for p in np.asarray(centres, dtype=np.float64):
        lo = np.floor(p - radius).astype(int)
        hi = np.floor(p + radius).astype(int)
        ix = np.arange(lo[0], hi[0] + 1)
        iy = np.arange(lo[1], hi[1] + 1)
        iz = np.arange(lo[2], hi[2] + 1)
        IZ, IY, IX = np.meshgrid(iz, iy, ix, indexing="ij")
        # nearest and farthest point of each cell to the centre
        dn = np.stack([np.clip(p[0], IX, IX + 1) - p[0],
                       np.clip(p[1], IY, IY + 1) - p[1],
                       np.clip(p[2], IZ, IZ + 1) - p[2]])
        dmin2 = np.einsum("a...,a...->...", dn, dn)
        fx = np.maximum(np.abs(IX - p[0]), np.abs(IX + 1 - p[0]))
        fy = np.maximum(np.abs(IY - p[1]), np.abs(IY + 1 - p[1]))
        fz = np.maximum(np.abs(IZ - p[2]), np.abs(IZ + 1 - p[2]))
        dmax2 = fx * fx + fy * fy + fz * fz
        full = dmax2 <= r2
        cut = (dmin2 < r2) & ~full
        wz, wy, wx = IZ % nz, IY % ny, IX % nx
        c[wz[full], wy[full], wx[full]] += 1.0
        if np.any(cut):
            cut_idx.append(np.stack([wz[cut], wy[cut], wx[cut]], axis=1))
            cut_geo.append(np.stack([IX[cut] - p[0], IY[cut] - p[1], IZ[cut] - p[2]], axis=1))
    if cut_idx:
        idx = np.concatenate(cut_idx)
        geo = np.concatenate(cut_geo)  # cell low corner relative to the centre
        chunk = 65536
        vals = np.empty(len(idx))
        for s in range(0, len(idx), chunk):
            g = geo[s:s + chunk]
            x = g[:, 0:1] + QX[None, :]
            y = g[:, 1:2] + QY[None, :]
            hw = np.sqrt(np.maximum(r2 - x * x - y * y, 0.0))
            z0 = g[:, 2:3]
            seg = np.clip(np.minimum(z0 + 1.0, hw) - np.maximum(z0, -hw), 0.0, 1.0)
            vals[s:s + chunk] = seg @ QW
        np.add.at(c, (idx[:, 0], idx[:, 1], idx[:, 2]), vals)
    np.clip(c, 0.0, 1.0, out=c)
    if not inside:
        c = 1.0 - c
    return c


# ---------------------------------------------------------------------------
# colour assignment of drops at t = 0


def conflict_distance(radius, w):
    """Centre distance below which two spheres may meet the near-contact test.

    A sphere occupies cells whose centres lie within radius + sqrt(3)/2 of its
    centre, and the (2w+1)^3 stencil test pairs cells whose centre offset is
    2*delta with |delta|_inf <= w, i.e. at most 2*w*sqrt(3) apart.
    """
    return 2.0 * radius + math.sqrt(3.0) * (1.0 + 2.0 * w) + 1.0


def greedy_colours(shape, centres, radius, w):
    """Colour spheres so that spheres closer than :func:`conflict_distance`
    never share a colour (DSatur greedy: repeatedly colour the uncoloured
    sphere with the most distinct neighbour colours, ties to the higher
    degree, then to the lower index, with the smallest free colour).
    Returns an int array of colours 0.. and the number of colours used."""
    L = np.array([shape[2], shape[1], shape[0]], dtype=np.float64)
    P = np.asarray(centres, dtype=np.float64)
    n = len(P)
    if n == 0:
        return np.zeros(0, dtype=np.int64), 0
    dc = conflict_distance(radius, w)
    adj = []
    for i in range(n):
        d = P - P[i]
        d -= L * np.round(d / L)
        nb = np.nonzero(np.einsum("ij,ij->i", d, d) < dc * dc)[0]
        adj.append(nb[nb != i])
    deg = np.array([len(a) for a in adj], dtype=np.int64)
    colours = -np.ones(n, dtype=np.int64)
    used_mask = np.zeros(n, dtype=object)
    used_mask[:] = 0
    sat = np.zeros(n, dtype=np.int64)
    for _ in range(n):
        key = np.where(colours < 0, sat * (n + 1) * 4 + deg, -1)
        best = key.max()
        v = int(np.nonzero(key == best)[0][0])
        k = 0
        while (used_mask[v] >> k) & 1:
            k += 1
        colours[v] = k
        for u in adj[v]:
            if not (used_mask[u] >> k) & 1:
                used_mask[u] |= 1 << k
                sat[u] += 1
    return colours, int(colours.max()) + 1


def coloured_fields(shape, centres, radius, colours, k_capacity, **kw):
    """c[K][nz][ny][nx] with every sphere placed in the field of its colour."""
    c = np.zeros((k_capacity,) + tuple(shape), dtype=np.float64)
    for k in range(int(colours.max()) + 1 if len(colours) else 0):
        sel = centres[colours == k]
        if len(sel):
            c[k] = sphere_cell_fractions(shape, sel, radius, **kw)
    return c


# ---------------------------------------------------------------------------
# velocity


def solenoidal_velocity(shape, n_modes, amplitude, drift, seed, h=1.0, vertical_axis=2):
    """Discretely divergence-free face velocity u[3][nz][ny][nx].

    A vector potential psi = sum_m a_m sin(2 pi k_m . x / L + phi_m) with integer
    wave vectors k_m in [-3, 3]^3 \\ {0}, random phases and random unit
    amplitudes a_m orthogonal to k_m is sampled on cell edges; the face
    velocities are its discrete curl (edge differences / h), so the discrete
    divergence of every cell vanishes up to round-off.  The random part is
    scaled so that its largest face speed equals ``amplitude``; a uniform
    ``drift`` along ``vertical_axis`` is added.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-3, 4, size=3)
        if np.any(k != 0):
            ks.append(k.astype(np.float64))
    ks = np.array(ks)
    phases = rng.random(n_modes) * 2.0 * math.pi
    amps = []
    for k in ks:
        v = rng.normal(size=3)
        kk = k / np.linalg.norm(k)
        v -= (v @ kk) * kk
        amps.append(v / np.linalg.norm(v))
    amps = np.array(amps)
    Ldim = np.array([nx, ny, nz], dtype=np.float64)

    def psi_component(comp, off):
        # sample component ``comp`` of psi at positions (i+off0, j+off1, k+off2)
        out = np.zeros(shape, dtype=np.float64)
        xs = (np.arange(nx) + off[0]) / Ldim[0]
        ys = (np.arange(ny) + off[1]) / Ldim[1]
        zs = (np.arange(nz) + off[2]) / Ldim[2]
        for m in range(n_modes):
            if amps[m, comp] == 0.0:
                continue
            ex = np.exp(2j * math.pi * ks[m, 0] * xs)
            ey = np.exp(2j * math.pi * ks[m, 1] * ys)
            ez = np.exp(2j * math.pi * ks[m, 2] * zs)
            ph = np.exp(1j * phases[m])
            val = (ph * ez)[:, None, None] * ey[None, :, None] * ex[None, None, :]
            out += amps[m, comp] * val.imag
        return out

    X = psi_component(0, (0.5, 0.0, 0.0))   # psi_x at (i+1/2, j, k)
    Y = psi_component(1, (0.0, 0.5, 0.0))   # psi_y at (i, j+1/2, k)
    Z = psi_component(2, (0.0, 0.0, 0.5))   # psi_z at (i, j, k+1/2)

    def sh(a, axis):  # a[... index+1 ...] with periodic wrap
        return np.roll(a, -1, axis=axis)

    ux = (sh(Z, 1) - Z) - (sh(Y, 0) - Y)
    uy = (sh(X, 0) - X) - (sh(Z, 2) - Z)
    uz = (sh(Y, 2) - Y) - (sh(X, 1) - X)
    u = np.stack([ux, uy, uz]) / h
    umax = np.abs(u).max()
    if umax > 0 and amplitude > 0:
        u *= amplitude / umax
    else:
        u[...] = 0.0
    u[vertical_axis] += drift
    return u


def uniform_velocity(shape, vec):
    u = np.zeros((3,) + tuple(shape), dtype=np.float64)
    for d in range(3):
        u[d] = vec[d]
    return u


def dt_for_cfl(u, cfl, h=1.0):
    """Time step such that max_faces |u_d| dt / h = cfl."""
    umax = float(np.abs(u).max())
    return cfl * h / umax if umax > 0 else 0.0


# ---------------------------------------------------------------------------
# named workloads


@dataclass
class Workload:
    name: str
    shape: tuple
    k_capacity: int
    k_active: int
    c: np.ndarray          # float64 [K][nz][ny][nx]
    u: np.ndarray          # float64 [3][nz][ny][nx]
    dt: float
    h: float
    steps: int
    radius: float
    centres: np.ndarray
    colours: np.ndarray
    stencil_w: int = 2


def make_workload(name, n=None, k_capacity=None, phi=None, radius=8.0, n_modes=16,
                  amplitude=0.5, drift=1.0, cfl=0.3, steps=1, seed=0, w=2,
                  n_spheres=None, shape=None):
    """Spheres at volume fraction ``phi`` (or ``n_spheres``), greedily coloured
    over fields, plus a seeded solenoidal velocity and the CFL time step."""
    if shape is None:
        shape = (n, n, n)
    if n_spheres is None:
        n_spheres = n_spheres_for_phi(shape, radius, phi)
    centres = rsa_centres(shape, radius, n_spheres, seed)
    colours, used = greedy_colours(shape, centres, radius, w)
    if k_capacity is None:
        k_capacity = max(used, 1)
    if used > k_capacity:
        raise ValueError(f"initial colouring needs {used} fields > capacity {k_capacity}")
    c = coloured_fields(shape, centres, radius, colours, k_capacity)
    u = solenoidal_velocity(shape, n_modes, amplitude, drift, seed + 1000)
    dt = dt_for_cfl(u, cfl)
    return Workload(name, tuple(shape), k_capacity, max(used, 1), c, u, dt, 1.0,
                    steps, radius, centres, colours, w)


def config_small(seed=1):
    """32^3, K = 1, 8 spheres of radius 4, u = (0,0,1) + 4 modes of amplitude
    0.2, CFL 0.25, 20 steps (no recolouring)."""
    shape = (32, 32, 32)
    centres = rsa_centres(shape, 4.0, 8, seed)
    colours = np.zeros(8, dtype=np.int64)
    c = coloured_fields(shape, centres, 4.0, colours, 1)
    u = solenoidal_velocity(shape, 4, 0.2, 1.0, seed + 1000)
    return Workload("32^3 K=1 8 spheres r=4", shape, 1, 1, c, u,
                    dt_for_cfl(u, 0.25), 1.0, 20, 4.0, centres, colours)


def config_medium(seed=2):
    """128^3, phi = 0.1 (98 spheres of radius 8), K = 4 with recolouring,
    16 modes of amplitude 0.5 plus vertical drift 1, CFL 0.3, 200 steps."""
    wl = make_workload("128^3 K=4 phi=0.1 r=8", n=128, k_capacity=4, phi=0.1,
                       radius=8.0, n_modes=16, amplitude=0.5, drift=1.0, cfl=0.3,
                       steps=200, seed=seed)
    return wl


def config_large(seed=3, k_capacity=8):
    """256^3, phi = 0.3 (2347 spheres of radius 8), K = 8, same velocity
    family, CFL 0.3, 100 steps."""
    return make_workload("256^3 K=8 phi=0.3 r=8", n=256, k_capacity=k_capacity, phi=0.3,
                         radius=8.0, n_modes=16, amplitude=0.5, drift=1.0, cfl=0.3,
                         steps=100, seed=seed)


def batched_specs(seed=5, n_boxes=64, sizes=(32, 48, 64, 96, 128)):
    """(edge n, phi, K drawn) of each box of the batched workload, in order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_boxes):
        n = int(rng.choice(sizes))
        phi = float(rng.uniform(0.05, 0.3))
        k = int(rng.integers(2, 9))
        out.append((n, phi, k))
    return out


def config_batched(seed=5, n_boxes=64, sizes=(32, 48, 64, 96, 128), select=None):
    """Independent tri-periodic boxes: edge drawn from ``sizes``, phi uniform
    in [0.05, 0.3], K uniform in [2, 8] (raised to the number of fields the
    initial colouring needs), spheres of radius 4 cells in boxes under 64
    cells and 8 cells otherwise, 16-mode solenoidal velocity of amplitude 0.5
    plus a vertical drift of 1, CFL 0.3.  Returns a list of Workloads: every
    box, or the boxes whose indices are in ``select`` (each box is the same
    whichever others are built)."""
    out = []
    for b, (n, phi, k) in enumerate(batched_specs(seed, n_boxes, sizes)):
        if select is not None and b not in select:
            continue
        r = 4.0 if n < 64 else 8.0
        shape = (n, n, n)
        ns = n_spheres_for_phi(shape, r, phi)
        centres = rsa_centres(shape, r, ns, seed * 1000 + b)
        colours, used = greedy_colours(shape, centres, r, 2)
        K = max(k, int(used))
        c = coloured_fields(shape, centres, r, colours, K)
        u = solenoidal_velocity(shape, 16, 0.5, 1.0, seed * 1000 + b + 500)
        out.append(Workload(f"box {b}: {n}^3 K={K} phi={phi:.3f} r={r:g}", shape, K, int(used), c, u,
                            dt_for_cfl(u, 0.3), 1.0, 1, r, centres, colours))
    return out
