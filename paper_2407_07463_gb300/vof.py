"""Thin ctypes binding of libvof.so (the C ABI in include/vof.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and the stream.  There is no
fallback: if libvof.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvof.so")

VOF_OK = 0
VOF_ERR_ARG, VOF_ERR_CUDA, VOF_ERR_WORKSPACE, VOF_ERR_NO_FREE_FIELD = -1, -2, -3, -4
VOF_ERR_CFL, VOF_ERR_TIMEOUT, VOF_ERR_STATE, VOF_ERR_NONFINITE, VOF_ERR_CAPACITY = -5, -6, -7, -8, -9
VOF_FP64, VOF_MIXED, VOF_MIXED_LEARNED = 0, 1, 2

STATUS = {0: "VOF_OK", -1: "VOF_ERR_ARG", -2: "VOF_ERR_CUDA", -3: "VOF_ERR_WORKSPACE",
          -4: "VOF_ERR_NO_FREE_FIELD", -5: "VOF_ERR_CFL", -6: "VOF_ERR_TIMEOUT",
          -7: "VOF_ERR_STATE", -8: "VOF_ERR_NONFINITE", -9: "VOF_ERR_CAPACITY"}


class VofError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        extra = ""
        if status == -2 and _lib is not None:
            extra = f" ({_lib.vof_last_cuda_error().decode()})"
        super().__init__(f"{where}: {STATUS.get(status, status)}{extra}")


class vof_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("k_capacity", C.c_int32), ("k_active", C.c_int32), ("precision", C.c_int32),
                ("h", C.c_double), ("stencil_w", C.c_int32), ("connectivity", C.c_int32),
                ("tag_tau", C.c_double), ("alpha_fp64_band", C.c_double),
                ("recolour", C.c_int32), ("vertical_axis", C.c_int32),
                ("stats_rbins", C.c_int32), ("stats_tbins", C.c_int32), ("stats_dr", C.c_double),
                ("stats_every", C.c_int32)]


class vof_step_report(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("clipped_volume", C.c_double),
                ("n_active", C.c_int32), ("n_moved", C.c_int32),
                ("near_contact_steps", C.c_int32), ("field_steps", C.c_int64),
                ("faces_network", C.c_int64), ("faces_myc", C.c_int64), ("faces_myc_judged", C.c_int64),
                ("n_in_use", C.c_int32), ("n_in_use_max", C.c_int32)]


class vof_box_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("k_capacity", C.c_int32),
                ("k_active", C.c_int32), ("c_dev", C.c_void_p), ("u_dev", C.c_void_p), ("dt", C.c_double)]


class vof_batch_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("h", C.c_double), ("tag_tau", C.c_double),
                ("alpha_fp64_band", C.c_double), ("use_graph", C.c_int32), ("autotune", C.c_int32)]


class vof_batch_report_t(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("n_boxes", C.c_int32), ("cell_fields_per_step", C.c_int64),
                ("clipped_volume", C.c_double * 64), ("faces_network", C.c_int64), ("faces_myc", C.c_int64),
                ("faces_myc_judged", C.c_int64),
                ("update_warps", C.c_int32), ("update_blocks_per_sm", C.c_int32),
                ("tune_candidates", C.c_int32), ("tune_best_ms", C.c_float), ("graph_launches", C.c_int64),
                ("direct_steps", C.c_int64)]


class vof_train_params(C.Structure):
    _fields_ = [("n_train", C.c_int64), ("n_test", C.c_int64), ("epochs", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_float), ("seed", C.c_uint64),
                ("plane_fraction", C.c_float), ("r_min", C.c_float), ("r_max", C.c_float)]


class vof_train_report(C.Structure):
    _fields_ = [("final_loss", C.c_float), ("steps", C.c_int32),
                ("test_mean_deg_mlp", C.c_double), ("test_mean_deg_myc", C.c_double),
                ("test_p95_deg_mlp", C.c_double), ("test_p95_deg_myc", C.c_double),
                ("test_mean_deg_combined", C.c_double), ("test_p95_deg_combined", C.c_double),
                ("test_network_share", C.c_double), ("bin_count", C.c_int64 * 5),
                ("bin_mean_deg_mlp", C.c_double * 5), ("bin_mean_deg_myc", C.c_double * 5),
                ("bin_mean_deg_combined", C.c_double * 5)]


class vof_stats_out(C.Structure):
    _fields_ = [("n_drops", C.c_int32), ("d", C.c_double), ("n_p", C.c_double),
                ("volume", C.c_double), ("events", C.c_double), ("M", C.c_double * 3),
                ("R", C.c_double * 9), ("A", C.c_double * 9), ("chi_mean", C.c_double),
                ("chi_max", C.c_double), ("chi_drops", C.c_double)]


_lib = None

EXPORTS = ["vof_config_default", "vof_workspace_size", "vof_init", "vof_set_velocity", "vof_step",
           "vof_near_contact", "vof_label", "vof_recolour", "vof_stats", "vof_drop_table",
           "vof_pair_stats", "vof_plic_volume", "vof_plic_alpha", "vof_normals",
           "vof_state_size", "vof_get_state", "vof_set_state", "vof_launch_count",
           "vof_status_string", "vof_destroy", "vof_profile_enable", "vof_profile_read",
           "vof_profile_class_name", "vof_label_noalloc", "vof_mlp_weights_size",
           "vof_mlp_forward", "vof_tc_gemm_check", "vof_mlp_train_params_default",
           "vof_mlp_train_workspace_size", "vof_mlp_train", "vof_mlp_grad",
           "vof_mlp_params_to_weights", "vof_set_mlp", "vof_learned_normals",
           "vof_batch_config_default", "vof_batch_workspace_size", "vof_batch_init", "vof_batch_set_mlp",
           "vof_batch_tune", "vof_batch_step", "vof_batch_report", "vof_batch_destroy",
           "vof_last_cuda_error", "vof_wait_selftest", "vof_drop_shape", "vof_curvature",
           "vof_surface_tension"]


def lib():
    """Load libvof.so (raises if it was not built: no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    cfgp = C.POINTER(vof_config)
    sig = {
        "vof_config_default": (C.c_int, [cfgp]),
        "vof_workspace_size": (C.c_size_t, [cfgp]),
        "vof_init": (C.c_int, [cfgp, vp, vp, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "vof_set_velocity": (C.c_int, [vp, vp]),
        "vof_step": (C.c_int, [vp, dbl, i32, C.POINTER(vof_step_report)]),
        "vof_near_contact": (C.c_int, [vp, vp]),
        "vof_label": (C.c_int, [vp, i32, vp, C.POINTER(i32)]),
        "vof_recolour": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32)]),
        "vof_stats": (C.c_int, [vp, i32, C.POINTER(vof_stats_out), vp, vp]),
        "vof_drop_table": (C.c_int, [vp, i32, vp, i32, vp, vp]),
        "vof_drop_shape": (C.c_int, [vp, i32, vp, i32, vp, vp, vp]),
        "vof_curvature": (C.c_int, [vp, i32, vp]),
        "vof_surface_tension": (C.c_int, [vp, dbl, vp]),
        "vof_pair_stats": (C.c_int, [vp, i64, vp, i32, i32, dbl, i32, dbl, dbl, vp, vp, vp, vp]),
        "vof_plic_volume": (C.c_int, [i32, vp, vp, vp, i64, vp]),
        "vof_plic_alpha": (C.c_int, [i32, vp, vp, vp, i64, dbl, vp]),
        "vof_normals": (C.c_int, [vp, i32, vp]),
        "vof_state_size": (C.c_size_t, [vp]),
        "vof_get_state": (C.c_int, [vp, vp, C.c_size_t]),
        "vof_set_state": (C.c_int, [vp, vp, C.c_size_t]),
        "vof_launch_count": (C.c_int64, [vp]),
        "vof_status_string": (C.c_char_p, [C.c_int]),
        "vof_destroy": (None, [vp]),
        "vof_profile_enable": (C.c_int, [vp, i32]),
        "vof_profile_read": (C.c_int, [vp, vp, vp, i32]),
        "vof_profile_class_name": (C.c_char_p, [i32]),
        "vof_label_noalloc": (C.c_int, [vp, i32, i32, i32, i32, dbl, i32, vp, C.POINTER(i32), vp]),
        "vof_mlp_weights_size": (C.c_size_t, []),
        "vof_mlp_forward": (C.c_int, [vp, vp, vp, i64, vp]),
        "vof_tc_gemm_check": (C.c_int, [vp, vp, vp, i32, i32, i32, vp]),
        "vof_mlp_train_params_default": (C.c_int, [C.POINTER(vof_train_params)]),
        "vof_mlp_train_workspace_size": (C.c_size_t, [C.POINTER(vof_train_params)]),
        "vof_mlp_train": (C.c_int, [C.POINTER(vof_train_params), vp, vp, C.c_size_t, vp,
                                    C.POINTER(vof_train_report)]),
        "vof_mlp_grad": (C.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "vof_mlp_params_to_weights": (C.c_int, [vp, vp, vp]),
        "vof_set_mlp": (C.c_int, [vp, vp, dbl]),
        "vof_learned_normals": (C.c_int, [vp, vp, i64, dbl, vp, vp, vp]),
        "vof_batch_config_default": (C.c_int, [C.POINTER(vof_batch_config)]),
        "vof_batch_workspace_size": (C.c_size_t, [C.POINTER(vof_batch_config), C.POINTER(vof_box_desc), i32]),
        "vof_batch_init": (C.c_int, [C.POINTER(vof_batch_config), C.POINTER(vof_box_desc), i32, vp, C.c_size_t,
                                     vp, C.POINTER(vp)]),
        "vof_batch_set_mlp": (C.c_int, [vp, vp, dbl]),
        "vof_batch_tune": (C.c_int, [vp]),
        "vof_batch_step": (C.c_int, [vp, i32]),
        "vof_batch_report": (C.c_int, [vp, C.POINTER(vof_batch_report_t)]),
        "vof_batch_destroy": (None, [vp]),
        "vof_last_cuda_error": (C.c_char_p, []),
        "vof_wait_selftest": (C.c_int, [i64, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return _lib


def _check(status, where):
    if status != VOF_OK:
        raise VofError(status, where)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_config(nx, ny, nz, k_capacity=1, k_active=1, precision=VOF_FP64, **kw):
    cfg = vof_config()
    _check(lib().vof_config_default(C.byref(cfg)), "vof_config_default")
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.k_capacity, cfg.k_active, cfg.precision = k_capacity, k_active, precision
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


def vof_workspace_size(cfg):
    return int(lib().vof_workspace_size(C.byref(cfg)))


# --------------------------------------------------------------------------- stateless


def vof_plic_volume(m, alpha, precision=VOF_FP64, stream=None):
    import torch
    v = torch.empty_like(alpha)
    _check(lib().vof_plic_volume(precision, _ptr(m), _ptr(alpha), _ptr(v), alpha.numel(),
                                 _stream(stream)), "vof_plic_volume")
    return v


def vof_plic_alpha(m, c, precision=VOF_FP64, band=1e-3, stream=None):
    import torch
    a = torch.empty_like(c)
    _check(lib().vof_plic_alpha(precision, _ptr(m), _ptr(c), _ptr(a), c.numel(), float(band),
                                _stream(stream)), "vof_plic_alpha")
    return a


def vof_pair_stats(cen, box, n_rbins, dr, n_tbins=150, dtheta=np.pi / 150, tie_tol=0.0,
                   vertical_axis=2, hist_r=None, hist_rt=None, moments=None, stream=None):
    """Accumulate nearest-particle statistics of centroids cen[n][3] (double,
    on the GPU); returns (hist_r, hist_rt, moments) device tensors."""
    import torch
    dev = cen.device
    if hist_r is None:
        hist_r = torch.zeros(n_rbins + 1, dtype=torch.float64, device=dev)
        hist_rt = torch.zeros((n_rbins + 1) * n_tbins, dtype=torch.float64, device=dev)
        moments = torch.zeros(13, dtype=torch.float64, device=dev)
    boxa = (C.c_double * 3)(*[float(b) for b in box])
    _check(lib().vof_pair_stats(_ptr(cen), cen.shape[0], C.cast(boxa, C.c_void_p), vertical_axis,
                                n_rbins, float(dr), n_tbins, float(dtheta), float(tie_tol),
                                _ptr(hist_r), _ptr(hist_rt), _ptr(moments), _stream(stream)),
           "vof_pair_stats")
    return hist_r, hist_rt, moments


def vof_label_noalloc(c, precision=VOF_FP64, tag_tau=0.0, connectivity=6, out=None, stream=None):
    """Tags of one field c[nz][ny][nx] (device tensor) through the entry point
    that allocates nothing inside the library; returns (labels, n)."""
    import torch
    nz, ny, nx = c.shape
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.int32, device=c.device)
    n = C.c_int32()
    _check(lib().vof_label_noalloc(_ptr(c), precision, nx, ny, nz, float(tag_tau), connectivity,
                                   _ptr(out), C.byref(n), _stream(stream)), "vof_label_noalloc")
    return out, n.value


def vof_mlp_forward(weights, stencils, stream=None):
    """Normals [n][3] of raw stencils [n][27] (float32 device tensors)."""
    import torch
    n = stencils.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=stencils.device)
    _check(lib().vof_mlp_forward(_ptr(weights), _ptr(stencils), _ptr(out), n, _stream(stream)),
           "vof_mlp_forward")
    return out


MLP_NPARAM = 64 * 32 + 64 * 64 + 16 * 64 + 64 + 64 + 16


def mlp_weights_empty(device="cuda"):
    import torch
    return torch.zeros(int(lib().vof_mlp_weights_size()), dtype=torch.uint8, device=device)


def vof_mlp_params_to_weights(params, weights=None, stream=None):
    """Flat FP32 parameters (device tensor, 7312 values) -> weight blob."""
    if weights is None:
        weights = mlp_weights_empty(params.device)
    _check(lib().vof_mlp_params_to_weights(_ptr(params), _ptr(weights), _stream(stream)),
           "vof_mlp_params_to_weights")
    return weights


def mlp_weights_to_params(weights):
    """Weight blob (device or host bytes) -> the flat parameters W1[64][32],
    W2[64][64], W3[16][64], b1[64], b2[64], b3[16] as float64 (7312 values;
    the BF16 weights are exact in float64).  Host-side unpacking only."""
    raw = np.asarray(weights.cpu().numpy() if hasattr(weights, "cpu") else weights, dtype=np.uint8)
    nw = 64 * 32 + 64 * 64 + 16 * 64
    if raw.size != 2 * nw + 4 * (64 + 64 + 16):
        raise ValueError("not a weight blob")
    w16 = raw[:2 * nw].view(np.uint16).astype(np.uint32) << np.uint32(16)
    out = np.empty(MLP_NPARAM)
    out[:nw] = w16.view(np.float32)
    out[nw:] = raw[2 * nw:].view(np.float32)
    return out


def vof_mlp_grad(weights, stencils, targets, stream=None):
    import torch
    g = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=stencils.device)
    loss = torch.zeros(1, dtype=torch.float32, device=stencils.device)
    _check(lib().vof_mlp_grad(_ptr(weights), _ptr(stencils), _ptr(targets), stencils.shape[0], _ptr(g),
                              _ptr(loss), _stream(stream)), "vof_mlp_grad")
    return g, float(loss.item())


def train_params(**kw):
    tp = vof_train_params()
    _check(lib().vof_mlp_train_params_default(C.byref(tp)), "vof_mlp_train_params_default")
    for k, v in kw.items():
        setattr(tp, k, v)
    return tp


def vof_mlp_train(tp, device="cuda", stream=None):
    """Train on the GPU; returns (weight blob tensor, report dict)."""
    import torch
    nbytes = int(lib().vof_mlp_train_workspace_size(C.byref(tp)))
    if nbytes == 0:
        raise VofError(-1, "vof_mlp_train_workspace_size")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    w = mlp_weights_empty(device)
    rep = vof_train_report()
    _check(lib().vof_mlp_train(C.byref(tp), _ptr(w), _ptr(ws), nbytes, _stream(stream), C.byref(rep)),
           "vof_mlp_train")
    del ws
    out = {}
    for k, _ in vof_train_report._fields_:
        v = getattr(rep, k)
        out[k] = list(v) if k.startswith("bin_") else v
    return w, out


def vof_learned_normals(weights, stencils, fallback_tol=1e-3, stream=None):
    """Judged learned normals of float stencils [n][27] (device); returns
    (normals [n][3] float, which [n] int32: 0 network, 1 MYC)."""
    import torch
    n = stencils.shape[0]
    m = torch.empty((n, 3), dtype=torch.float32, device=stencils.device)
    which = torch.empty(n, dtype=torch.int32, device=stencils.device)
    _check(lib().vof_learned_normals(_ptr(weights), _ptr(stencils), n, float(fallback_tol), _ptr(m),
                                     _ptr(which), _stream(stream)), "vof_learned_normals")
    return m, which


def vof_wait_selftest(poll_limit=100000, stream=None):
    """Runs the bounded-wait self-test; returns its status (VOF_ERR_TIMEOUT
    expected)."""
    return lib().vof_wait_selftest(int(poll_limit), _stream(stream))


def vof_tc_gemm_check(a, b, variant=0, stream=None):
    import torch
    n, k = b.shape
    d = torch.empty((128, n), dtype=torch.float32, device=a.device)
    _check(lib().vof_tc_gemm_check(_ptr(a), _ptr(b), _ptr(d), k, n, variant, _stream(stream)),
           "vof_tc_gemm_check")
    return d


# --------------------------------------------------------------------------- context


class Context:
    """One context per set of borrowed buffers (c [K][nz][ny][nx], u [3][nz][ny][nx])."""

    def __init__(self, cfg, c, u, stream=None):
        import torch
        self.cfg = cfg
        self.c = c
        self.u = u
        dt = torch.float64 if cfg.precision == VOF_FP64 else torch.float32
        if c.dtype != dt or u.dtype != dt:
            raise TypeError(f"c and u must be {dt}")
        if tuple(c.shape) != (cfg.k_capacity, cfg.nz, cfg.ny, cfg.nx) or not c.is_contiguous():
            raise ValueError("c must be contiguous [K][nz][ny][nx]")
        if tuple(u.shape) != (3, cfg.nz, cfg.ny, cfg.nx) or not u.is_contiguous():
            raise ValueError("u must be contiguous [3][nz][ny][nx]")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = vof_workspace_size(cfg)
        if nbytes == 0:
            raise VofError(-1, "vof_workspace_size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=c.device)
        h = C.c_void_p()
        _check(lib().vof_init(C.byref(cfg), _ptr(c), _ptr(u), _ptr(self.workspace), nbytes,
                              _stream(self.stream), C.byref(h)), "vof_init")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().vof_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vof_step(self, dt, nsteps=1, report=True):
        rep = vof_step_report()
        st = lib().vof_step(self.handle, float(dt), int(nsteps), C.byref(rep) if report else None)
        if st not in (VOF_OK, VOF_ERR_NO_FREE_FIELD):
            raise VofError(st, "vof_step")
        if not report:
            return None
        return {"status": st, "steps_done": rep.steps_done, "clipped_volume": rep.clipped_volume,
                "n_active": rep.n_active, "n_moved": rep.n_moved,
                "near_contact_steps": rep.near_contact_steps, "field_steps": rep.field_steps,
                "faces_network": rep.faces_network, "faces_myc": rep.faces_myc,
                "faces_myc_judged": rep.faces_myc_judged, "n_in_use": rep.n_in_use,
                "n_in_use_max": rep.n_in_use_max}

    step = vof_step

    def vof_set_mlp(self, weights, fallback_tol=1e-3):
        """Borrow a device weight blob (uint8 tensor of vof_mlp_weights_size()
        bytes) for the learned normal; it must outlive its use."""
        self.mlp_weights = weights
        _check(lib().vof_set_mlp(self.handle, _ptr(weights), float(fallback_tol)), "vof_set_mlp")

    def vof_set_velocity(self, u):
        self.u = u
        _check(lib().vof_set_velocity(self.handle, _ptr(u)), "vof_set_velocity")

    def vof_near_contact(self):
        flags = (C.c_int32 * self.cfg.k_capacity)()
        _check(lib().vof_near_contact(self.handle, C.cast(flags, C.c_void_p)), "vof_near_contact")
        return np.array(flags[:], dtype=np.int32)

    def vof_label(self, field, out=None):
        import torch
        if out is None:
            out = torch.empty((self.cfg.nz, self.cfg.ny, self.cfg.nx), dtype=torch.int32,
                              device=self.c.device)
        n = C.c_int32()
        _check(lib().vof_label(self.handle, int(field), _ptr(out), C.byref(n)), "vof_label")
        return out, n.value

    def vof_recolour(self):
        moved = C.c_int32()
        na = C.c_int32()
        st = lib().vof_recolour(self.handle, C.byref(moved), C.byref(na))
        if st not in (VOF_OK, VOF_ERR_NO_FREE_FIELD):
            raise VofError(st, "vof_recolour")
        return moved.value, na.value, st

    def vof_stats(self, reset=False, histograms=True):
        out = vof_stats_out()
        nr, nt = self.cfg.stats_rbins, self.cfg.stats_tbins
        hr = np.zeros(nr + 1) if histograms else None
        hrt = np.zeros((nr + 1) * nt) if histograms else None
        _check(lib().vof_stats(self.handle, int(bool(reset)), C.byref(out),
                               hr.ctypes.data_as(C.c_void_p) if histograms else None,
                               hrt.ctypes.data_as(C.c_void_p) if histograms else None),
               "vof_stats")
        res = {"n_drops": out.n_drops, "d": out.d, "n_p": out.n_p, "volume": out.volume,
               "events": out.events, "M": np.array(out.M[:]),
               "R": np.array(out.R[:]).reshape(3, 3), "A": np.array(out.A[:]).reshape(3, 3),
               "chi_mean": out.chi_mean, "chi_max": out.chi_max, "chi_drops": out.chi_drops}
        if histograms:
            res["hist_r"] = hr
            res["hist_rt"] = hrt.reshape(nr + 1, nt)
        return res

    def vof_drop_table(self, field, labels, n_labels):
        import torch
        vol = torch.zeros(max(n_labels, 1), dtype=torch.float64, device=self.c.device)
        cen = torch.zeros((max(n_labels, 1), 3), dtype=torch.float64, device=self.c.device)
        _check(lib().vof_drop_table(self.handle, int(field), _ptr(labels), int(n_labels), _ptr(vol),
                                    _ptr(cen)), "vof_drop_table")
        return vol[:n_labels], cen[:n_labels]

    def vof_drop_shape(self, field, labels, n_labels, cen):
        """(inertia [n][6] = xx yy zz xy xz yz, chi [n]) of the drops of a
        field given its labels and centroids (vof_drop_table)."""
        import torch
        inertia = torch.zeros((max(n_labels, 1), 6), dtype=torch.float64, device=self.c.device)
        chi = torch.zeros(max(n_labels, 1), dtype=torch.float64, device=self.c.device)
        _check(lib().vof_drop_shape(self.handle, int(field), _ptr(labels), int(n_labels),
                                    _ptr(cen.contiguous()), _ptr(inertia), _ptr(chi)), "vof_drop_shape")
        return inertia[:n_labels], chi[:n_labels]

    def vof_curvature(self, field, out=None):
        """Height-function curvature of one field (NaN where a cell has none)."""
        import torch
        if out is None:
            out = torch.empty((self.cfg.nz, self.cfg.ny, self.cfg.nx), dtype=self.c.dtype, device=self.c.device)
        _check(lib().vof_curvature(self.handle, int(field), _ptr(out)), "vof_curvature")
        return out

    def vof_surface_tension(self, gamma, out=None):
        """f[3][nz][ny][nx] = sum_i gamma kappa_i grad C_i on the low faces."""
        import torch
        if out is None:
            out = torch.empty((3, self.cfg.nz, self.cfg.ny, self.cfg.nx), dtype=self.c.dtype,
                              device=self.c.device)
        _check(lib().vof_surface_tension(self.handle, float(gamma), _ptr(out)), "vof_surface_tension")
        return out

    def vof_normals(self, field):
        import torch
        m = torch.empty((self.cfg.nz, self.cfg.ny, self.cfg.nx, 3), dtype=self.c.dtype,
                        device=self.c.device)
        _check(lib().vof_normals(self.handle, int(field), _ptr(m)), "vof_normals")
        return m

    def vof_get_state(self):
        n = int(lib().vof_state_size(self.handle))
        buf = np.zeros(n, dtype=np.uint8)
        _check(lib().vof_get_state(self.handle, buf.ctypes.data_as(C.c_void_p), n), "vof_get_state")
        return buf

    def vof_set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().vof_set_state(self.handle, buf.ctypes.data_as(C.c_void_p), buf.size),
               "vof_set_state")

    def vof_profile_enable(self, on=True):
        _check(lib().vof_profile_enable(self.handle, int(bool(on))), "vof_profile_enable")

    def vof_profile_read(self):
        """{class name: (launches, total ms)} of the launches recorded since the
        last read."""
        n = 32
        cnt = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        _check(lib().vof_profile_read(self.handle, C.cast(cnt, C.c_void_p), C.cast(ms, C.c_void_p), n),
               "vof_profile_read")
        out = {}
        for i in range(n):
            name = lib().vof_profile_class_name(i)
            if name is None:
                break
            if cnt[i]:
                out[name.decode()] = (int(cnt[i]), float(ms[i]))
        return out

    @property
    def launches(self):
        return int(lib().vof_launch_count(self.handle))


# --------------------------------------------------------------------------- batches


class Batch:
    """Independent boxes advanced together (one launch per sweep pass for
    every box, graph replay, tuned update launch shape).  boxes: list of
    (c, u, dt) with c [K][nz][ny][nx] and u [3][nz][ny][nx] device tensors
    of the precision's dtype; k_active: list or None (all fields)."""

    def __init__(self, boxes, precision=VOF_MIXED, k_active=None, h=1.0, tag_tau=1e-6, band=1e-3,
                 use_graph=True, autotune=True, stream=None):
        import torch
        cfg = vof_batch_config()
        _check(lib().vof_batch_config_default(C.byref(cfg)), "vof_batch_config_default")
        cfg.precision = precision
        cfg.h = h
        cfg.tag_tau = tag_tau
        cfg.alpha_fp64_band = band
        cfg.use_graph = 1 if use_graph else 0
        cfg.autotune = 1 if autotune else 0
        self.cfg = cfg
        self.boxes = boxes
        n = len(boxes)
        arr = (vof_box_desc * n)()
        for b, (c, u, dt) in enumerate(boxes):
            K, nz, ny, nx = c.shape
            arr[b].nx, arr[b].ny, arr[b].nz = nx, ny, nz
            arr[b].k_capacity = K
            arr[b].k_active = K if k_active is None else int(k_active[b])
            arr[b].c_dev = _ptr(c)
            arr[b].u_dev = _ptr(u)
            arr[b].dt = float(dt)
        self.desc = arr
        nbytes = int(lib().vof_batch_workspace_size(C.byref(cfg), arr, n))
        if nbytes == 0:
            raise VofError(VOF_ERR_ARG, "vof_batch_workspace_size")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=boxes[0][0].device)
        h_ = C.c_void_p()
        _check(lib().vof_batch_init(C.byref(cfg), arr, n, _ptr(self.workspace), nbytes, _stream(self.stream),
                                    C.byref(h_)), "vof_batch_init")
        self.handle = h_

    def set_mlp(self, weights, fallback_tol=1e-3):
        self.mlp_weights = weights
        _check(lib().vof_batch_set_mlp(self.handle, _ptr(weights), float(fallback_tol)), "vof_batch_set_mlp")

    def tune(self):
        _check(lib().vof_batch_tune(self.handle), "vof_batch_tune")

    def step(self, nsteps=1):
        _check(lib().vof_batch_step(self.handle, int(nsteps)), "vof_batch_step")

    def report(self):
        r = vof_batch_report_t()
        _check(lib().vof_batch_report(self.handle, C.byref(r)), "vof_batch_report")
        d = {k: getattr(r, k) for k, _ in vof_batch_report_t._fields_ if k != "clipped_volume"}
        d["clipped_volume"] = list(r.clipped_volume[:r.n_boxes])
        return d

    def close(self):
        if getattr(self, "handle", None):
            lib().vof_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
