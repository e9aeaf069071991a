"""FP64 CPU oracle of the multi-field VoF step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.
The C source (``oracle.c``) shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _compile(out, extra, force):
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force=False):
    """Compile liboracle.so with gcc (no FMA contraction, so every machine
    rounds the same way), and liboracle_omp.so, the same source with OpenMP
    (z-planes of the advection step in parallel; identical results).  The
    OpenMP build is skipped if the compiler lacks OpenMP."""
    _compile(_LIB, [], force)
    try:
        _compile(_LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return _LIB


def lib(omp=False):
    """The serial oracle, or (omp=True) its OpenMP build; None if that build
    is unavailable."""
    global _lib, _lib_omp
    with _lock:
        if omp:
            if _lib_omp is None:
                build()
                if not os.path.exists(_LIB_OMP):
                    return None
                _lib_omp = _declare(C.CDLL(_LIB_OMP))
            return _lib_omp
        if _lib is None:
            build()
            _lib = _declare(C.CDLL(_LIB))
    return _lib


def threads(n=0, omp=True):
    """Threads the OpenMP build uses (n > 0 sets them); 1 without it."""
    L = lib(omp=omp)
    return 1 if L is None else int(L.oracle_threads(int(n)))


def _declare(L):
    L.oracle_plic_volume.restype = C.c_double
    L.oracle_plic_volume.argtypes = [_dp, C.c_double]
    L.oracle_plic_alpha.restype = C.c_double
    L.oracle_plic_alpha.argtypes = [_dp, C.c_double]
    for f in ("oracle_youngs", "oracle_myc"):
        getattr(L, f).restype = None
        getattr(L, f).argtypes = [_dp, _dp]
    L.oracle_centred_column.restype = None
    L.oracle_centred_column.argtypes = [_dp, C.c_int, _dp]
    L.oracle_myc_choice.restype = C.c_int
    L.oracle_myc_choice.argtypes = [_dp]
    L.oracle_face_flux.restype = C.c_double
    L.oracle_face_flux.argtypes = [_dp, C.c_double, C.c_int, C.c_double]
    L.oracle_cell_face_flux.restype = C.c_double
    L.oracle_cell_face_flux.argtypes = [_dp] + [C.c_int] * 7 + [C.c_double]
    L.oracle_advect_step.restype = C.c_int
    L.oracle_advect_step.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_double, C.c_double, C.c_int64, _dp]
    L.oracle_normals.restype = None
    L.oracle_normals.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp]
    L.oracle_label.restype = C.c_int64
    L.oracle_label.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _ip]
    L.oracle_near_contact.restype = C.c_int
    L.oracle_near_contact.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
    L.oracle_near_contact_map.restype = None
    L.oracle_near_contact_map.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_double, _up]
    L.oracle_near_pairs.restype = C.c_int64
    L.oracle_near_pairs.argtypes = [_dp, _ip, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.c_void_p, C.c_void_p, C.c_int64]
    L.oracle_recolour.restype = C.c_int
    L.oracle_recolour.argtypes = [_dp, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                  C.c_int, C.c_int, C.c_double, C.c_int,
                                  C.POINTER(C.c_int), C.c_void_p, C.c_int]
    L.oracle_drop_table.restype = None
    L.oracle_drop_table.argtypes = [_dp, _ip, C.c_int64, C.c_int, C.c_int, C.c_int,
                                    C.c_double, _dp, _dp]
    L.oracle_pair_stats.restype = None
    L.oracle_pair_stats.argtypes = [_dp, C.c_int64, _dp, C.c_int, C.c_int, C.c_double,
                                    C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp,
                                    _dp]
    L.oracle_canon.restype = None
    L.oracle_canon.argtypes = [_dp, _dp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.oracle_mlp_forward.restype = None
    L.oracle_mlp_forward.argtypes = [_dp, _dp, C.c_int, _dp]
    L.oracle_normal_residual.restype = C.c_double
    L.oracle_normal_residual.argtypes = [_dp, _dp]
    L.oracle_learned_normal.restype = C.c_int
    L.oracle_learned_normal.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_int, _dp,
                                        C.POINTER(C.c_int)]
    L.oracle_advect_step_learned.restype = C.c_int
    L.oracle_advect_step_learned.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.c_double, C.c_int64, _dp,
                                             C.c_double, C.c_double, C.c_int, _dp,
                                             C.POINTER(C.c_int64), C.c_void_p]
    L.oracle_mlp_loss_grad.restype = C.c_double
    L.oracle_mlp_loss_grad.argtypes = [_dp, _dp, _dp, C.c_int64, C.c_int, _dp]
    L.oracle_drop_inertia.restype = None
    L.oracle_drop_inertia.argtypes = [_dp, _ip, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_double, _dp,
                                      _dp, _dp]
    L.oracle_curvature.restype = None
    L.oracle_curvature.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp]
    L.oracle_curvature_along.restype = None
    L.oracle_curvature_along.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, _dp]
    L.oracle_surface_tension.restype = None
    L.oracle_surface_tension.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                         C.c_double, _dp]
    L.oracle_threads.restype = C.c_int
    L.oracle_threads.argtypes = [C.c_int]
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------- PLIC


def plic_volume(m, alpha):
    return lib().oracle_plic_volume(_f64(m), float(alpha))


def plic_alpha(m, c):
    return lib().oracle_plic_alpha(_f64(m), float(c))


def youngs(st):
    out = np.zeros(3)
    lib().oracle_youngs(_f64(st).ravel(), out)
    return out


def centred_column(st, axis):
    out = np.zeros(3)
    lib().oracle_centred_column(_f64(st).ravel(), int(axis), out)
    return out


def myc(st):
    out = np.zeros(3)
    lib().oracle_myc(_f64(st).ravel(), out)
    return out


def myc_choice(st):
    return lib().oracle_myc_choice(_f64(st).ravel())


def face_flux(m, alpha, d, s):
    return lib().oracle_face_flux(_f64(m), float(alpha), int(d), float(s))


def cell_face_flux(c, i, j, k, d, s):
    nz, ny, nx = c.shape
    return lib().oracle_cell_face_flux(_f64(c), nx, ny, nz, i, j, k, d, float(s))


# --------------------------------------------------------------------------- advection


def advect_step(c, u, dt, h, step_index, omp=False):
    """One step of every field; returns (c_new, clipped[K]).  omp=True runs
    the OpenMP build (same result)."""
    c = np.array(c, dtype=np.float64, order="C", copy=True)
    squeeze = c.ndim == 3
    if squeeze:
        c = c[None]
    K, nz, ny, nx = c.shape
    clipped = np.zeros(K)
    rc = ((lib(omp=True) if omp else None) or lib()).oracle_advect_step(
        c, _f64(u), nx, ny, nz, K, float(dt), float(h), int(step_index), clipped)
    if rc != 0:
        raise MemoryError("oracle_advect_step")
    return (c[0] if squeeze else c), clipped


def advect_step_learned(c, u, dt, h, step_index, params, tol=1e-3, amb_eps=1e-6, amb_choice=0,
                        amb_map=None, omp=False):
    """One step with the learned normal (MYC fallback); returns (c_new,
    clipped[K], counts) with counts = (faces on the network, on MYC,
    ambiguous decisions resolved by amb_choice).  amb_map (uint8 array of
    c's shape, optional) gets 1 on both cells of every ambiguous face."""
    c = np.array(c, dtype=np.float64, order="C", copy=True)
    squeeze = c.ndim == 3
    if squeeze:
        c = c[None]
    K, nz, ny, nx = c.shape
    clipped = np.zeros(K)
    counts = (C.c_int64 * 3)()
    L = (lib(omp=True) if omp else None) or lib()
    rc = L.oracle_advect_step_learned(c, _f64(u), nx, ny, nz, K, float(dt), float(h),
                                          int(step_index), _f64(params), float(tol), float(amb_eps),
                                          int(amb_choice), clipped, counts,
                                          None if amb_map is None else amb_map.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_advect_step_learned")
    return (c[0] if squeeze else c), clipped, tuple(counts)


def normal_residual(st, n):
    """Mean residual over the 27 cells of the plane of normal n through the
    centre cell (judge of the learned normal)."""
    return lib().oracle_normal_residual(_f64(np.asarray(st).reshape(27)), _f64(n))


def learned_normal(params, st, tol=1e-3, amb_eps=0.0, amb_choice=0):
    """(m, which, ambiguous): L1-normalised normal, 0 = network / 1 = MYC."""
    m = np.zeros(3)
    amb = C.c_int(0)
    which = lib().oracle_learned_normal(_f64(params), _f64(np.asarray(st).reshape(27)), float(tol),
                                        float(amb_eps), int(amb_choice), m, C.byref(amb))
    return m, which, amb.value


def advect(c, u, dt, h, steps, first_step=0, omp=False):
    clipped = 0.0
    for s in range(steps):
        c, cl = advect_step(c, u, dt, h, first_step + s, omp=omp)
        clipped = clipped + cl
    return c, clipped


def normals(c):
    nz, ny, nx = c.shape
    out = np.zeros((nz, ny, nx, 3))
    lib().oracle_normals(_f64(c), nx, ny, nz, out)
    return out


def curvature(c, h=1.0):
    """Height-function curvature of every cell of one field (NaN where none)."""
    nz, ny, nx = c.shape
    out = np.zeros(c.shape)
    lib().oracle_curvature(_f64(c), nx, ny, nz, float(h), out)
    return out


def curvature_along(c, axis, sign, h=1.0):
    """Curvature with the height columns along `axis` and the c = 1 phase at
    the -sign end, for every interfacial cell (NaN where a column misses the
    interface)."""
    nz, ny, nx = c.shape
    out = np.zeros(c.shape)
    lib().oracle_curvature_along(_f64(c), nx, ny, nz, float(h), int(axis), int(sign), out)
    return out


def surface_tension(c, kappa, gamma=1.0, h=1.0):
    """f[3][nz][ny][nx] = sum_i gamma kappa_i grad C_i on the low faces."""
    c = _f64(c)
    if c.ndim == 3:
        c = c[None]
    kappa = _f64(kappa).reshape(c.shape)
    K, nz, ny, nx = c.shape
    f = np.zeros((3, nz, ny, nx))
    lib().oracle_surface_tension(c, kappa, K, nx, ny, nz, float(h), float(gamma), f)
    return f


# --------------------------------------------------------------------------- tagging


def label(c, tau=0.0, connectivity=6):
    nz, ny, nx = c.shape
    lab = np.zeros(c.shape, dtype=np.int32)
    n = lib().oracle_label(_f64(c), nx, ny, nz, float(tau), int(connectivity), lab)
    if n < 0:
        raise MemoryError("oracle_label")
    return lab, int(n)


def near_contact(c, w=2, tau=0.0):
    nz, ny, nx = c.shape
    return bool(lib().oracle_near_contact(_f64(c), nx, ny, nz, int(w), float(tau)))


def near_contact_map(c, w=2, tau=0.0):
    nz, ny, nx = c.shape
    out = np.zeros(c.shape, dtype=np.uint8)
    lib().oracle_near_contact_map(_f64(c), nx, ny, nz, int(w), float(tau), out)
    return out


def near_pairs(c, lab, w=2, tau=0.0):
    nz, ny, nx = c.shape
    cf = _f64(c)
    lb = np.ascontiguousarray(lab, dtype=np.int32)
    n = lib().oracle_near_pairs(cf, lb, nx, ny, nz, int(w), float(tau), None, None, 0)
    pa = np.zeros(max(n, 1), dtype=np.int32)
    pb = np.zeros(max(n, 1), dtype=np.int32)
    lib().oracle_near_pairs(cf, lb, nx, ny, nz, int(w), float(tau),
                            pa.ctypes.data, pb.ctypes.data, n)
    return np.stack([pa[:n], pb[:n]], axis=1)


def recolour(c, n_active, w=2, tau=0.0, connectivity=6, log_cap=4096):
    """Steps 1-4; returns (c_new, n_active, n_moved, status, moves[(field,label,target)])."""
    c = np.array(c, dtype=np.float64, order="C", copy=True)
    K, nz, ny, nx = c.shape
    na = C.c_int(int(n_active))
    nm = C.c_int(0)
    log = np.full((log_cap, 3), -1, dtype=np.int32)
    st = lib().oracle_recolour(c, K, C.byref(na), nx, ny, nz, int(w), float(tau),
                               int(connectivity), C.byref(nm), log.ctypes.data, log_cap)
    if st == -1:
        raise MemoryError("oracle_recolour")
    moves = log[: min(nm.value, log_cap)]
    return c, na.value, nm.value, st, moves


# --------------------------------------------------------------------------- statistics


def drop_table(c, lab, n_labels, h=1.0):
    nz, ny, nx = c.shape
    vol = np.zeros(max(n_labels, 1))
    cen = np.zeros((max(n_labels, 1), 3))
    lib().oracle_drop_table(_f64(c), np.ascontiguousarray(lab, dtype=np.int32), int(n_labels),
                            nx, ny, nz, float(h), vol, cen)
    return vol[:n_labels], cen[:n_labels]


def drop_inertia(c, lab, n_labels, cen=None, h=1.0):
    """(inertia[n][6] = xx yy zz xy xz yz, chi[n]) of the drops of one field
    (Appendix A); centroids from drop_table unless given."""
    nz, ny, nx = c.shape
    if cen is None:
        _, cen = drop_table(c, lab, n_labels, h)
    I = np.zeros((max(n_labels, 1), 6))
    chi = np.zeros(max(n_labels, 1))
    lib().oracle_drop_inertia(_f64(c), np.ascontiguousarray(lab, dtype=np.int32), int(n_labels), nx, ny, nz,
                              float(h), _f64(np.asarray(cen).reshape(-1, 3) if n_labels else np.zeros((1, 3))),
                              I, chi)
    return I[:n_labels], chi[:n_labels]


class PairStats:
    """Accumulators of the nearest-particle statistics (Section 3)."""

    def __init__(self, n_rbins, dr, n_tbins=150, dtheta=np.pi / 150):
        self.n_rbins, self.dr, self.n_tbins, self.dtheta = n_rbins, dr, n_tbins, dtheta
        self.hist_r = np.zeros(n_rbins + 1)
        self.hist_rt = np.zeros((n_rbins + 1) * n_tbins)
        self.msum = np.zeros(3)
        self.rsum = np.zeros(9)
        self.events = np.zeros(1)

    def add(self, cen, box, vertical_axis=2, tie_tol=0.0):
        cen = _f64(cen).reshape(-1, 3)
        lib().oracle_pair_stats(cen, len(cen), _f64(box), int(vertical_axis), self.n_rbins,
                                float(self.dr), self.n_tbins, float(self.dtheta),
                                float(tie_tol), self.hist_r, self.hist_rt, self.msum,
                                self.rsum, self.events)
        return self

    @property
    def E(self):
        return float(self.events[0])

    @property
    def M(self):
        return self.msum / self.E

    @property
    def R(self):
        return self.rsum.reshape(3, 3) / self.E

    @property
    def A(self):
        R = self.R
        return R - np.trace(R) / 3.0 * np.eye(3)


# --------------------------------------------------------------------------- learned normal

MLP_NPARAM = 64 * 32 + 64 * 64 + 16 * 64 + 64 + 64 + 16


def mlp_canon(st):
    """(x[27], sign[3], perm[3]) of a stencil st[3][3][3] ([k][j][i])."""
    x = np.zeros(27)
    sg = (C.c_int * 3)()
    pm = (C.c_int * 3)()
    lib().oracle_canon(_f64(st).ravel(), x, sg, pm)
    return x, list(sg), list(pm)


def mlp_forward(params, x, bf16=True):
    """Canonical-frame output.  bf16=True: BF16 weights and BF16 (hi, lo)
    layer inputs, as the tensor cores see them; bf16="weights": BF16 weights,
    FP64 layer inputs; False: all FP64."""
    mode = 2 if bf16 == "weights" else int(bool(bf16))
    out = np.zeros(3)
    lib().oracle_mlp_forward(_f64(params), _f64(x), mode, out)
    return out


def mlp_normal(params, st, bf16=True):
    """Network normal of a raw stencil, mapped back and L2-normalised."""
    x, sg, pm = mlp_canon(st)
    oc = mlp_forward(params, x, bf16)
    n = np.zeros(3)
    for q in range(3):
        n[pm[q]] = sg[pm[q]] * oc[q]
    return n / np.linalg.norm(n)


def mlp_loss_grad(params, x, t, bf16=True):
    x = _f64(x).reshape(-1, 27)
    t = _f64(t).reshape(-1, 3)
    g = np.zeros(MLP_NPARAM)
    loss = lib().oracle_mlp_loss_grad(_f64(params), x, t, len(x), int(bool(bf16)), g)
    return loss, g
