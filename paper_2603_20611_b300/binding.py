"""Thin ctypes binding of ``libgaussianpile.so`` (the C ABI in ``include/gp.h``).

Argument marshalling only: every function below checks tensor placement and
layout, passes raw device pointers and the current CUDA stream to the C entry
point of the same name, and raises ``GPError`` on a non-zero status.  There is
no fallback: if the shared library is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes
import lzma
import os
import struct

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GP_LIBRARY=check selects the bounds-checked debug build (see build.py)
LIB_PATH = os.path.join(_HERE, "libgaussianpile_check.so" if os.environ.get("GP_LIBRARY") == "check"
                        else "libgaussianpile.so")

GP_OK = 0
GP_PENDING = 1
GP_ERR_ARG = -1
GP_ERR_OOM = -2
GP_ERR_CUDA = -3
GP_ERR_TIMEOUT = -4
GP_ERR_OVERFLOW = -5
GP_ERR_STATE = -6
GP_ERR_CANCELLED = -7
GP_EXP_POLY = 0
GP_EXP_HW = 1
GP_EXP_POLY_PACKED = 2
GP_EXP_POLY_ROW = 3
GP_EXP_POLY_GRAD = 4
GP_EXP_POLY_GRAD_PACKED = 5

# Every symbol include/gp.h declares (checked by the CPU ABI test).
EXPORTS = (
    "gp_config_default", "gp_create", "gp_destroy", "gp_last_error", "gp_workspace_bytes",
    "gp_render_slices", "gp_render_backward", "gp_mse_grad", "gp_voxelize", "gp_voxelize_backward",
    "gp_last_counts", "gp_count_evals", "gp_exp2_eval", "gp_timing_enable", "gp_timing_enable_phases",
    "gp_timing_read",
    "gp_launch_count", "gp_fma_probe_threads", "gp_fma_probe", "gp_mse_grad_noalloc",
    "gp_batch_plan", "gp_batch_run", "gp_batch_wait", "gp_batch_info", "gp_batch_destroy",
    "gp_serve_open", "gp_serve_load_set", "gp_serve_submit", "gp_serve_poll", "gp_serve_cancel", "gp_serve_stats_get",
    "gp_serve_close", "gp_view_from_axis", "gp_render_slices_view", "gp_render_backward_view",
    "gp_count_evals_view", "gp_adam_default", "gp_adam_state_floats", "gp_adam_init", "gp_adam_step",
    "gp_l1_dssim_grad", "gp_encode", "gp_decode", "gp_serve_load_encoded", "gp_count_vox_evals",
    "gp_fma_probe_mode", "gp_fma_probe_lane_fmas", "gp_check_enabled", "gp_check_selftest",
    "gp_count_evaluated_view", "gp_count_vox_evaluated",
)
GP_REQ_SLICE, GP_REQ_STACK, GP_REQ_VOXELIZE = 0, 1, 2
GP_RASTER_AUTO, GP_RASTER_BLOCK, GP_RASTER_ROWS, GP_RASTER_PIXELS = 0, 1, 2, 3
GP_BATCH_AUTOTUNE = 1
GP_NUM_PHASES = 8
PHASES = ("bin", "fwd", "bwd", "bwd_pre", "loss", "vox_fwd", "vox_bwd", "opt")


class GPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class gp_config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("deterministic", ctypes.c_int), ("exp_mode", ctypes.c_int),
                ("tile", ctypes.c_int), ("fwd_px", ctypes.c_int), ("bwd_px", ctypes.c_int),
                ("workspace_limit", ctypes.c_int64), ("reuse_bins", ctypes.c_int), ("raster", ctypes.c_int)]


class gp_set(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("n", ctypes.c_int64), ("scale_mod", ctypes.c_float)]


class gp_view(ctypes.Structure):
    """Slice orientation [R_c | t]: camera coordinates x_c = R x + t (R row-major)."""
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3)]


def make_view(view):
    """A gp_view from a gp_view or an (R [3, 3], t [3]) pair."""
    if isinstance(view, gp_view):
        return view
    R, t = view
    R = np.asarray(R, np.float32).reshape(9)
    t = np.asarray(t, np.float32).reshape(3)
    return gp_view((ctypes.c_float * 9)(*R.tolist()), (ctypes.c_float * 3)(*t.tolist()))


class gp_batch_item(ctypes.Structure):
    _fields_ = [("set", gp_set), ("z", ctypes.c_void_p), ("S", ctypes.c_int), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("sigma_z", ctypes.c_float), ("axis", ctypes.c_int),
                ("out", ctypes.c_void_p), ("target", ctypes.c_void_p), ("dL_dI", ctypes.c_void_p),
                ("d_mu", ctypes.c_void_p), ("d_scale", ctypes.c_void_p), ("d_quat", ctypes.c_void_p),
                ("d_alpha", ctypes.c_void_p), ("loss", ctypes.c_void_p), ("view", ctypes.c_void_p)]


class gp_batch_config(ctypes.Structure):
    _fields_ = [("pair_capacity", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("tile", ctypes.c_int),
                ("fwd_raster", ctypes.c_int), ("bwd_raster", ctypes.c_int), ("fwd_chunk", ctypes.c_int),
                ("bwd_chunk", ctypes.c_int), ("fwd_px", ctypes.c_int), ("bwd_px", ctypes.c_int)]


class gp_codec_header(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos_bits", ctypes.c_int), ("lo", ctypes.c_float * 3),
                ("hi", ctypes.c_float * 3), ("log_s_min", ctypes.c_double), ("log_s_max", ctypes.c_double)]


class gp_adam_cfg(ctypes.Structure):
    _fields_ = [("lr_mu", ctypes.c_float), ("lr_scale", ctypes.c_float), ("lr_quat", ctypes.c_float),
                ("lr_alpha", ctypes.c_float), ("mu_extent", ctypes.c_float), ("lr_final_ratio", ctypes.c_float),
                ("total_steps", ctypes.c_int64), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("log_scale_logit_alpha", ctypes.c_int)]


class gp_serve_cfg(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("max_batch_slices", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_int64), ("hbm_reserve_bytes", ctypes.c_int64)]


class gp_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("set_id", ctypes.c_int), ("z", ctypes.c_void_p), ("S", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("sigma_z", ctypes.c_float), ("axis", ctypes.c_int),
                ("X", ctypes.c_int), ("Y", ctypes.c_int), ("Z", ctypes.c_int), ("out", ctypes.c_void_p),
                ("view", ctypes.c_void_p), ("timeout_ms", ctypes.c_double)]


class gp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("batch_size", ctypes.c_int)]


class gp_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "batches", "admission_waits",
                                              "pending", "inflight_bytes", "inflight_requests",
                                              "max_inflight_requests", "expired", "cancelled")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2603_20611_b300.build` "
                          "(the operator has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    CP, SP = ctypes.POINTER(gp_config), ctypes.POINTER(gp_set)
    sig = {
        "gp_config_default": [CP],
        "gp_create": [ctypes.POINTER(P), I, CP],
        "gp_destroy": [P],
        "gp_last_error": [P],
        "gp_workspace_bytes": [P],
        "gp_render_slices": [P, SP, P, I, I, I, F, I, P, P],
        "gp_render_backward": [P, SP, P, I, I, I, F, I, P, P, P, P, P, P],
        "gp_mse_grad": [P, P, P, P, I, I, I, P, P, P],
        "gp_voxelize": [P, SP, I, I, I, P, P],
        "gp_voxelize_backward": [P, SP, I, I, I, P, P, P, P, P, P],
        "gp_last_counts": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "gp_count_evals": [P, SP, P, I, I, I, F, I, ctypes.POINTER(I64)],
        "gp_exp2_eval": [P, P, P, I64, I, P],
        "gp_timing_enable": [P, I],
        "gp_timing_enable_phases": [P, ctypes.c_uint],
        "gp_timing_read": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "gp_launch_count": [],
        "gp_fma_probe_threads": [P],
        "gp_fma_probe": [P, I, P, P],
        "gp_fma_probe_mode": [P, I, I, P, P],
        "gp_fma_probe_lane_fmas": [I],
        "gp_check_enabled": [],
        "gp_check_selftest": [P, P],
        "gp_mse_grad_noalloc": [P, P, P, I, I, I, P, P, P],
        "gp_batch_plan": [P, ctypes.POINTER(gp_batch_item), I, I, ctypes.POINTER(P)],
        "gp_batch_run": [P, P],
        "gp_batch_wait": [P, P],
        "gp_batch_info": [P, ctypes.POINTER(gp_batch_config)],
        "gp_batch_destroy": [P],
        "gp_serve_open": [P, ctypes.POINTER(gp_serve_cfg), ctypes.POINTER(P)],
        "gp_serve_load_set": [P, SP, ctypes.POINTER(I)],
        "gp_serve_submit": [P, ctypes.POINTER(gp_request), ctypes.POINTER(ctypes.c_uint64)],
        "gp_serve_poll": [P, ctypes.c_uint64, I, ctypes.POINTER(gp_result)],
        "gp_serve_cancel": [P, ctypes.c_uint64],
        "gp_serve_stats_get": [P, ctypes.POINTER(gp_serve_stats)],
        "gp_serve_close": [P],
        "gp_view_from_axis": [I, ctypes.POINTER(gp_view)],
        "gp_render_slices_view": [P, SP, ctypes.POINTER(gp_view), P, I, I, I, F, P, P],
        "gp_render_backward_view": [P, SP, ctypes.POINTER(gp_view), P, I, I, I, F, P, P, P, P, P, P],
        "gp_count_evals_view": [P, SP, ctypes.POINTER(gp_view), P, I, I, I, F, ctypes.POINTER(I64)],
        "gp_count_evaluated_view": [P, SP, ctypes.POINTER(gp_view), P, I, I, I, F, ctypes.POINTER(I64),
                                    ctypes.POINTER(I64)],
        "gp_count_vox_evaluated": [P, SP, I, I, I, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "gp_adam_default": [ctypes.POINTER(gp_adam_cfg)],
        "gp_l1_dssim_grad": [P, P, P, P, I, I, I, F, P, P, P],
        "gp_encode": [P, SP, I, ctypes.POINTER(gp_codec_header), P, P, P],
        "gp_count_vox_evals": [P, SP, I, I, I, ctypes.POINTER(I64)],
        "gp_decode": [P, ctypes.POINTER(gp_codec_header), P, P, P, P, P, P],
        "gp_serve_load_encoded": [P, ctypes.POINTER(gp_codec_header), P, F, ctypes.POINTER(I)],
        "gp_adam_state_floats": [I64],
        "gp_adam_init": [P, ctypes.POINTER(gp_adam_cfg), I64, P, P, P, P],
        "gp_adam_step": [P, ctypes.POINTER(gp_adam_cfg), I64, I64, P, P, P, P, P, P, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.gp_last_error.restype = ctypes.c_char_p
    lib.gp_workspace_bytes.restype = I64
    lib.gp_launch_count.restype = I64
    lib.gp_fma_probe_threads.restype = I64
    lib.gp_adam_state_floats.restype = I64
    return lib


lib = _load()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, name, dtype=torch.float32, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host_f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1))


class Context:
    """Owns a gp_ctx (device workspace pool) on one CUDA device."""

    def __init__(self, device=0, eps=1e-6, deterministic=False, exp_mode=GP_EXP_POLY, tile=16,
                 fwd_px=0, bwd_px=0, workspace_limit=0, reuse_bins=False, raster=None):
        cfg = gp_config()
        lib.gp_config_default(ctypes.byref(cfg))
        cfg.eps, cfg.deterministic, cfg.exp_mode = float(eps), int(bool(deterministic)), int(exp_mode)
        cfg.tile, cfg.fwd_px, cfg.bwd_px = int(tile), int(fwd_px), int(bwd_px)
        cfg.workspace_limit = int(workspace_limit)
        cfg.reuse_bins = int(bool(reuse_bins))
        if raster is not None:
            cfg.raster = int(raster)
        self.device = int(device)
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = lib.gp_create(ctypes.byref(h), self.device, ctypes.byref(cfg))
        if st != GP_OK:
            raise GPError(st, "gp_create failed")
        self.h = h

    def check(self, st, what):
        if st != GP_OK:
            msg = lib.gp_last_error(self.h).decode(errors="replace")
            raise GPError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self):
        return int(lib.gp_workspace_bytes(self.h))

    def timing(self, enable=True, phases=None):
        """Phase timing on (all phases, or only the named ones) or off."""
        if phases is None or not enable:
            self.check(lib.gp_timing_enable(self.h, int(bool(enable))), "gp_timing_enable")
        else:
            mask = 0
            for p in phases:
                mask |= 1 << PHASES.index(p)
            self.check(lib.gp_timing_enable_phases(self.h, mask), "gp_timing_enable_phases")

    def timing_read(self):
        """{phase: (ms, launches, calls)} since the last read."""
        ms = (ctypes.c_double * GP_NUM_PHASES)()
        ln = (ctypes.c_int64 * GP_NUM_PHASES)()
        cl = (ctypes.c_int64 * GP_NUM_PHASES)()
        self.check(lib.gp_timing_read(self.h, ms, ln, cl), "gp_timing_read")
        return {PHASES[k]: (ms[k], ln[k], cl[k]) for k in range(GP_NUM_PHASES)}

    def fma_probe(self, iters, out=None, stream=None, mode=0):
        """Launch the throughput probe; returns (out, lane operations it performs).
        mode 0: scalar FFMA chains, 1: packed FFMA2 chains, 2: both mixed,
        3: chains of the SFU ex2.approx instruction."""
        n = int(lib.gp_fma_probe_threads(self.h))
        if out is None:
            out = torch.empty(n, device=f"cuda:{self.device}")
        self.check(lib.gp_fma_probe_mode(self.h, int(mode), int(iters), _dev(out, "out", shape=(n,)),
                                         _stream(stream)), "gp_fma_probe_mode")
        return out, n * int(iters) * int(lib.gp_fma_probe_lane_fmas(int(mode)))

    def last_counts(self):
        p, e = ctypes.c_int64(), ctypes.c_int64()
        self.check(lib.gp_last_counts(self.h, ctypes.byref(p), ctypes.byref(e)), "gp_last_counts")
        return int(p.value), int(e.value)


class GaussianSet:
    """Device tensors of one Gaussian set (Sec. S1: G = (mu, s, q, alpha))."""

    def __init__(self, mu, scale, quat, alpha, scale_mod=1.0):
        self.mu, self.scale, self.quat, self.alpha = mu, scale, quat, alpha
        self.scale_mod = float(scale_mod)

    @property
    def n(self):
        return int(self.alpha.shape[0])

    @classmethod
    def from_numpy(cls, g, device="cuda", scale_mod=1.0):
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return cls(f(g.mu), f(g.scale), f(g.quat), f(g.alpha), scale_mod)

    def c(self):
        n = self.n
        return gp_set(_dev(self.mu, "mu", shape=(n, 3)).value, _dev(self.scale, "scale", shape=(n, 3)).value,
                      _dev(self.quat, "quat", shape=(n, 4)).value, _dev(self.alpha, "alpha", shape=(n,)).value,
                      n, self.scale_mod)


def _grads_like(gs, grads):
    n = gs.n
    if grads is None:
        dev = gs.alpha.device
        grads = (torch.empty(n, 3, device=dev), torch.empty(n, 3, device=dev), torch.empty(n, 4, device=dev),
                 torch.empty(n, device=dev))
    return grads


def view_from_axis(axis):
    v = gp_view()
    st = lib.gp_view_from_axis(int(axis), ctypes.byref(v))
    if st != GP_OK:
        raise GPError(st, "gp_view_from_axis")
    return v


def gp_render_slices(ctx, gs, z, H, W, sigma_z, axis=2, out=None, stream=None, view=None):
    """view (a gp_view or (R, t)) selects a general slice orientation; axis is then ignored."""
    z = _host_f32(z)
    S = z.shape[0]
    if out is None:
        out = torch.empty(S, H, W, device=gs.alpha.device)
    zp = z.ctypes.data_as(ctypes.c_void_p)
    o = _dev(out, "out", shape=(S, H, W))
    if view is not None:
        v = make_view(view)
        st = lib.gp_render_slices_view(ctx.h, ctypes.byref(gs.c()), ctypes.byref(v), zp, S, H, W, float(sigma_z),
                                       o, _stream(stream))
    else:
        st = lib.gp_render_slices(ctx.h, ctypes.byref(gs.c()), zp, S, H, W, float(sigma_z), axis, o,
                                  _stream(stream))
    ctx.check(st, "gp_render_slices")
    return out


def gp_render_backward(ctx, gs, z, H, W, sigma_z, dL_dI, axis=2, grads=None, stream=None, view=None):
    z = _host_f32(z)
    S = z.shape[0]
    d_mu, d_s, d_q, d_a = _grads_like(gs, grads)
    zp = z.ctypes.data_as(ctypes.c_void_p)
    gargs = (_dev(dL_dI, "dL_dI", shape=(S, H, W)), _dev(d_mu, "d_mu"), _dev(d_s, "d_scale"),
             _dev(d_q, "d_quat"), _dev(d_a, "d_alpha"), _stream(stream))
    if view is not None:
        v = make_view(view)
        st = lib.gp_render_backward_view(ctx.h, ctypes.byref(gs.c()), ctypes.byref(v), zp, S, H, W,
                                         float(sigma_z), *gargs)
    else:
        st = lib.gp_render_backward(ctx.h, ctypes.byref(gs.c()), zp, S, H, W, float(sigma_z), axis, *gargs)
    ctx.check(st, "gp_render_backward")
    return d_mu, d_s, d_q, d_a


def gp_mse_grad(ctx, I, T, t_index=None, dL_dI=None, loss=None, stream=None):
    S, H, W = I.shape
    if dL_dI is None:
        dL_dI = torch.empty_like(I)
    tid = None
    if t_index is not None:
        tid = np.ascontiguousarray(np.asarray(t_index, np.int32).reshape(-1))
        if tid.shape[0] != S:
            raise ValueError("t_index needs one entry per slice")
        if T.dim() != 3 or T.shape[1:] != I.shape[1:] or int(tid.max(initial=0)) >= T.shape[0]:
            raise ValueError("target stack too small for t_index")
    elif tuple(T.shape) != tuple(I.shape):
        raise ValueError("T must match I when t_index is None")
    st = lib.gp_mse_grad(ctx.h, _dev(I, "I"), _dev(T, "T"),
                         None if tid is None else tid.ctypes.data_as(ctypes.c_void_p), S, H, W,
                         _dev(dL_dI, "dL_dI", shape=(S, H, W)),
                         None if loss is None else _dev(loss, "loss", shape=(1,)), _stream(stream))
    ctx.check(st, "gp_mse_grad")
    return dL_dI, loss


def gp_l1_dssim_grad(ctx, I, T, t_index=None, lam=0.2, dL_dI=None, loss=None, stream=None):
    """The paper's loss L1 + lam (1 - SSIM) and dL/dI; loss (3 floats, device)
    receives (L, L1, mean SSIM)."""
    S, H, W = I.shape
    if dL_dI is None:
        dL_dI = torch.empty_like(I)
    tid = None
    if t_index is not None:
        tid = np.ascontiguousarray(np.asarray(t_index, np.int32).reshape(-1))
        if tid.shape[0] != S or T.dim() != 3 or T.shape[1:] != I.shape[1:] or int(tid.max(initial=0)) >= T.shape[0]:
            raise ValueError("t_index needs one in-range entry per slice")
    elif tuple(T.shape) != tuple(I.shape):
        raise ValueError("T must match I when t_index is None")
    st = lib.gp_l1_dssim_grad(ctx.h, _dev(I, "I"), _dev(T, "T"),
                              None if tid is None else tid.ctypes.data_as(ctypes.c_void_p), S, H, W, float(lam),
                              _dev(dL_dI, "dL_dI", shape=(S, H, W)),
                              None if loss is None else _dev(loss, "loss", shape=(3,)), _stream(stream))
    ctx.check(st, "gp_l1_dssim_grad")
    return dL_dI, loss


def gp_mse_grad_noalloc(I, T, t_index=None, dL_dI=None, loss=None, stream=None):
    """gp_mse_grad without a context or any device allocation by the library
    (scratch is a fixed array inside the library; see include/gp.h)."""
    S, H, W = I.shape
    if dL_dI is None:
        dL_dI = torch.empty_like(I)
    tid = None
    if t_index is not None:
        tid = np.ascontiguousarray(np.asarray(t_index, np.int32).reshape(-1))
        if tid.shape[0] != S or int(tid.max(initial=0)) >= T.shape[0]:
            raise ValueError("t_index needs one in-range entry per slice")
    elif tuple(T.shape) != tuple(I.shape):
        raise ValueError("T must match I when t_index is None")
    st = lib.gp_mse_grad_noalloc(_dev(I, "I"), _dev(T, "T"),
                                 None if tid is None else tid.ctypes.data_as(ctypes.c_void_p), S, H, W,
                                 _dev(dL_dI, "dL_dI", shape=(S, H, W)),
                                 None if loss is None else _dev(loss, "loss", shape=(1,)), _stream(stream))
    if st != GP_OK:
        raise GPError(st, "gp_mse_grad_noalloc")
    return dL_dI, loss


class BatchPlan:
    """A captured batch of renders (gp_batch_plan); run() replays its graph.

    items: dicts with keys gs (GaussianSet), z, H, W, sigma_z, axis and any of
    out, target, dL_dI, grads (4-tuple of tensors), loss (1-element tensor)."""

    def __init__(self, ctx, items, autotune=False):
        self.ctx = ctx
        self._keep = []
        arr = (gp_batch_item * len(items))()
        for k, it in enumerate(items):
            gs = it["gs"]
            z = _host_f32(it["z"])
            self._keep.append(z)
            S, H, W = z.shape[0], int(it["H"]), int(it["W"])
            c = arr[k]
            c.set = gs.c()
            c.z = z.ctypes.data_as(ctypes.c_void_p).value
            c.S, c.H, c.W = S, H, W
            c.sigma_z = float(it["sigma_z"])
            c.axis = int(it.get("axis", 2))
            if it.get("view") is not None:
                v = make_view(it["view"])
                self._keep.append(v)
                c.view = ctypes.addressof(v)
            for key in ("out", "target", "dL_dI"):
                t = it.get(key)
                setattr(c, key, None if t is None else _dev(t, key, shape=(S, H, W)).value)
            g = it.get("grads")
            if g is not None:
                c.d_mu, c.d_scale, c.d_quat, c.d_alpha = [_dev(t, "grad").value for t in g]
            if it.get("loss") is not None:
                c.loss = _dev(it["loss"], "loss", shape=(1,)).value
            self._keep.append(it)
        h = ctypes.c_void_p()
        ctx.check(lib.gp_batch_plan(ctx.h, arr, len(items), GP_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)),
                  "gp_batch_plan")
        self.h = h

    def run(self, stream=None):
        self.ctx.check(lib.gp_batch_run(self.h, _stream(stream)), "gp_batch_run")

    def wait(self, stream=None):
        st = lib.gp_batch_wait(self.h, _stream(stream))
        if st != GP_OK:
            raise GPError(st, "gp_batch_wait: " + lib.gp_last_error(self.ctx.h).decode(errors="replace"))

    def info(self):
        c = gp_batch_config()
        self.ctx.check(lib.gp_batch_info(self.h, ctypes.byref(c)), "gp_batch_info")
        form = {GP_RASTER_BLOCK: "block", GP_RASTER_ROWS: "rows", GP_RASTER_PIXELS: "pixels"}
        return {"pair_capacity": c.pair_capacity, "tile": c.tile,
                "fwd_raster": form.get(c.fwd_raster, c.fwd_raster), "fwd_chunk": c.fwd_chunk, "fwd_px": c.fwd_px,
                "bwd_raster": form.get(c.bwd_raster, c.bwd_raster), "bwd_chunk": c.bwd_chunk, "bwd_px": c.bwd_px,
                "device_bytes": c.device_bytes}

    def close(self):
        if getattr(self, "h", None):
            lib.gp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """gp_serve_*: resident sets, asynchronous requests, poll for completion."""

    def __init__(self, ctx, workers=4, max_batch_slices=64, hbm_budget_bytes=0, hbm_reserve_bytes=4 << 30):
        cfg = gp_serve_cfg(workers, max_batch_slices, hbm_budget_bytes, hbm_reserve_bytes)
        h = ctypes.c_void_p()
        st = lib.gp_serve_open(ctx.h, ctypes.byref(cfg), ctypes.byref(h))
        if st != GP_OK:
            raise GPError(st, "gp_serve_open")
        self.h = h
        self._sets = []
        self._outs = {}

    def load_set(self, gs):
        self._sets.append(gs)
        sid = ctypes.c_int()
        st = lib.gp_serve_load_set(self.h, ctypes.byref(gs.c()), ctypes.byref(sid))
        if st != GP_OK:
            raise GPError(st, "gp_serve_load_set")
        return sid.value

    def load_encoded(self, hdr, streams, scale_mod=1.0):
        """Registers a set decoded by the server from gp_encode output (the server owns the memory)."""
        sid = ctypes.c_int()
        sc = streams.contiguous()
        st = lib.gp_serve_load_encoded(self.h, ctypes.byref(hdr), _dev(sc, "streams", torch.int16), float(scale_mod),
                                       ctypes.byref(sid))
        if st != GP_OK:
            raise GPError(st, "gp_serve_load_encoded")
        return sid.value

    def submit(self, kind, set_id, out, z=None, H=0, W=0, sigma_z=1.0, axis=2, X=0, Y=0, Z=0, view=None,
               timeout_ms=0.0):
        """Queues a request; timeout_ms > 0 drops it (status GP_ERR_TIMEOUT) if it
        has not started that long after the submit."""
        r = gp_request()
        r.kind, r.set_id = int(kind), int(set_id)
        zz = None
        if z is not None:
            zz = _host_f32(z)
            r.z, r.S = zz.ctypes.data_as(ctypes.c_void_p).value, zz.shape[0]
        r.H, r.W, r.sigma_z, r.axis = int(H), int(W), float(sigma_z), int(axis)
        r.X, r.Y, r.Z = int(X), int(Y), int(Z)
        r.timeout_ms = float(timeout_ms)
        r.out = _dev(out, "out").value
        v = None
        if view is not None:
            v = make_view(view)
            r.view = ctypes.addressof(v)
        t = ctypes.c_uint64()
        st = lib.gp_serve_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if st != GP_OK:
            raise GPError(st, "gp_serve_submit")
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """None while pending, else a dict with status and latencies."""
        res = gp_result()
        st = lib.gp_serve_poll(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res))
        if st == GP_PENDING:
            return None
        if st != GP_OK:
            raise GPError(st, "gp_serve_poll")
        self._outs.pop(ticket, None)
        return {"status": res.status, "latency_ms": res.latency_ms, "queue_ms": res.queue_ms,
                "batch_size": res.batch_size}

    def cancel(self, ticket):
        """Removes a still-queued request (its poll status becomes GP_ERR_CANCELLED);
        GPError with GP_ERR_STATE once it has started."""
        st = lib.gp_serve_cancel(self.h, ctypes.c_uint64(ticket))
        if st != GP_OK:
            raise GPError(st, "gp_serve_cancel")

    def stats(self):
        s = gp_serve_stats()
        lib.gp_serve_stats_get(self.h, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in gp_serve_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib.gp_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gp_voxelize(ctx, gs, X, Y, Z, vol=None, stream=None):
    if vol is None:
        vol = torch.empty(Z, Y, X, device=gs.alpha.device)
    st = lib.gp_voxelize(ctx.h, ctypes.byref(gs.c()), X, Y, Z, _dev(vol, "vol", shape=(Z, Y, X)),
                         _stream(stream))
    ctx.check(st, "gp_voxelize")
    return vol


def gp_voxelize_backward(ctx, gs, X, Y, Z, dL_dV, grads=None, stream=None):
    d_mu, d_s, d_q, d_a = _grads_like(gs, grads)
    st = lib.gp_voxelize_backward(ctx.h, ctypes.byref(gs.c()), X, Y, Z, _dev(dL_dV, "dL_dV", shape=(Z, Y, X)),
                                  _dev(d_mu, "d_mu"), _dev(d_s, "d_scale"), _dev(d_q, "d_quat"),
                                  _dev(d_a, "d_alpha"), _stream(stream))
    ctx.check(st, "gp_voxelize_backward")
    return d_mu, d_s, d_q, d_a


def gp_count_evals(ctx, gs, z, H, W, sigma_z, axis=2, view=None):
    z = _host_f32(z)
    out = ctypes.c_int64()
    zp = z.ctypes.data_as(ctypes.c_void_p)
    if view is not None:
        v = make_view(view)
        st = lib.gp_count_evals_view(ctx.h, ctypes.byref(gs.c()), ctypes.byref(v), zp, z.shape[0], H, W,
                                     float(sigma_z), ctypes.byref(out))
    else:
        st = lib.gp_count_evals(ctx.h, ctypes.byref(gs.c()), zp, z.shape[0], H, W, float(sigma_z), axis,
                                ctypes.byref(out))
    ctx.check(st, "gp_count_evals")
    return int(out.value)


def gp_count_vox_evals(ctx, gs, X, Y, Z):
    out = ctypes.c_int64()
    ctx.check(lib.gp_count_vox_evals(ctx.h, ctypes.byref(gs.c()), X, Y, Z, ctypes.byref(out)), "gp_count_vox_evals")
    return int(out.value)


def gp_count_evaluated(ctx, gs, z, H, W, sigma_z, axis=2, view=None):
    """(forward, backward) pixels the context's default rasterisers evaluate for this render."""
    z = _host_f32(z)
    out, outb = ctypes.c_int64(), ctypes.c_int64()
    if view is not None:
        v = make_view(view)
    else:
        v = gp_view()
        if lib.gp_view_from_axis(int(axis), ctypes.byref(v)) != GP_OK:
            raise ValueError("axis must be 0, 1 or 2")
    st = lib.gp_count_evaluated_view(ctx.h, ctypes.byref(gs.c()), ctypes.byref(v), z.ctypes.data_as(ctypes.c_void_p),
                                     z.shape[0], H, W, float(sigma_z), ctypes.byref(out), ctypes.byref(outb))
    ctx.check(st, "gp_count_evaluated_view")
    return int(out.value), int(outb.value)


def gp_count_vox_evaluated(ctx, gs, X, Y, Z):
    """(forward, backward) voxels the context's default rasterisers evaluate for a voxelize."""
    out, outb = ctypes.c_int64(), ctypes.c_int64()
    ctx.check(lib.gp_count_vox_evaluated(ctx.h, ctypes.byref(gs.c()), X, Y, Z, ctypes.byref(out),
                                         ctypes.byref(outb)), "gp_count_vox_evaluated")
    return int(out.value), int(outb.value)


def gp_exp2_eval(ctx, x, mode=GP_EXP_POLY, y=None, stream=None):
    if y is None:
        y = torch.empty_like(x)
    st = lib.gp_exp2_eval(ctx.h, _dev(x, "x"), _dev(y, "y", shape=x.shape), x.numel(), int(mode), _stream(stream))
    ctx.check(st, "gp_exp2_eval")
    return y


def gp_encode(ctx, gs, pos_bits=14, stream=None):
    """(header, streams [11, n] int16 tensor holding uint16 codes, order [n] int32
    tensor) of the paper's codec; streams are zigzag deltas in Morton order."""
    hdr = gp_codec_header()
    n = gs.n
    dev = gs.alpha.device
    streams = torch.empty(11, max(n, 1), dtype=torch.int16, device=dev)
    order = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ctx.check(lib.gp_encode(ctx.h, ctypes.byref(gs.c()), int(pos_bits), ctypes.byref(hdr),
                            _dev(streams, "streams", torch.int16), _dev(order, "order", torch.int32),
                            _stream(stream)), "gp_encode")
    return hdr, streams[:, :n], order[:n]


def gp_decode(ctx, hdr, streams, scale_mod=1.0, stream=None):
    """GaussianSet decoded from a header and device streams (Morton order)."""
    n = int(hdr.n)
    dev = streams.device
    quat = torch.empty(n, 4, device=dev)
    gs = GaussianSet(torch.empty(n, 3, device=dev), torch.empty(n, 3, device=dev), quat,
                     torch.empty(n, device=dev), scale_mod)
    st = streams.contiguous()
    ctx.check(lib.gp_decode(ctx.h, ctypes.byref(hdr), _dev(st, "streams", torch.int16), _dev(gs.mu, "mu"),
                            _dev(gs.scale, "scale"), _dev(gs.quat, "quat"), _dev(gs.alpha, "alpha"),
                            _stream(stream)), "gp_decode")
    return gs


_CODEC_HDR = struct.Struct("<qi3f3f2d")


def encode_bytes(ctx, gs, pos_bits=14):
    """The whole storage path: device quantisation and delta streams, then LZMA
    on the host over the header and the little-endian uint16 streams."""
    hdr, streams, _ = gp_encode(ctx, gs, pos_bits)
    raw = _CODEC_HDR.pack(hdr.n, hdr.pos_bits, *hdr.lo, *hdr.hi, hdr.log_s_min, hdr.log_s_max)
    body = streams.cpu().numpy().astype("<i2").tobytes()
    return lzma.compress(raw + body)


def decode_bytes(ctx, blob, device="cuda", scale_mod=1.0):
    """Inverse of encode_bytes: LZMA on the host, then the device decode."""
    raw = lzma.decompress(blob)
    n, bits, lx, ly, lz, hx, hy, hz, l0, l1 = _CODEC_HDR.unpack_from(raw)
    hdr = gp_codec_header(n, bits, (ctypes.c_float * 3)(lx, ly, lz), (ctypes.c_float * 3)(hx, hy, hz), l0, l1)
    streams = torch.from_numpy(np.frombuffer(raw, "<i2", offset=_CODEC_HDR.size).reshape(11, n).copy()).to(device)
    return hdr, gp_decode(ctx, hdr, streams, scale_mod)


class Adam:
    """The fit loop's parameter update on the device (gp_adam_*): Adam with the
    paper's learning rates, decaying exponentially, on log s and logit alpha by
    default.  Owns its [26, n] state tensor; step() updates a GaussianSet in place."""

    def __init__(self, ctx, gs, total_steps=30000, mu_extent=1.0, log_scale_logit_alpha=True, **rates):
        self.ctx = ctx
        self.cfg = gp_adam_cfg()
        lib.gp_adam_default(ctypes.byref(self.cfg))
        self.cfg.total_steps = int(total_steps)
        self.cfg.mu_extent = float(mu_extent)
        self.cfg.log_scale_logit_alpha = int(bool(log_scale_logit_alpha))
        for k, v in rates.items():
            setattr(self.cfg, k, float(v))
        self.n = gs.n
        self.state = torch.empty(int(lib.gp_adam_state_floats(self.n)), device=gs.alpha.device)
        self.t = 0
        ctx.check(lib.gp_adam_init(ctx.h, ctypes.byref(self.cfg), self.n, _dev(gs.scale, "scale"),
                                   _dev(gs.alpha, "alpha"), _dev(self.state, "state"), _stream(None)),
                  "gp_adam_init")

    def step(self, gs, grads, stream=None):
        self.t += 1
        d_mu, d_s, d_q, d_a = grads
        self.ctx.check(lib.gp_adam_step(self.ctx.h, ctypes.byref(self.cfg), self.t, self.n, _dev(gs.mu, "mu"),
                                        _dev(gs.scale, "scale"), _dev(gs.quat, "quat"), _dev(gs.alpha, "alpha"),
                                        _dev(d_mu, "d_mu"), _dev(d_s, "d_scale"), _dev(d_q, "d_quat"),
                                        _dev(d_a, "d_alpha"), _dev(self.state, "state"), _stream(stream)),
                       "gp_adam_step")


class SliceRender(torch.autograd.Function):
    """Differentiable slice projection: forward gp_render_slices, backward
    gp_render_backward (per-tile lists rebuilt, no per-pixel state kept)."""

    @staticmethod
    def forward(fctx, ctx, z, H, W, sigma_z, axis, scale_mod, view, mu, scale, quat, alpha):
        gs = GaussianSet(mu.contiguous(), scale.contiguous(), quat.contiguous(), alpha.contiguous(), scale_mod)
        v = None if view is None else make_view(view)
        fctx.meta = (ctx, _host_f32(z).copy(), H, W, sigma_z, axis, scale_mod, v)
        fctx.save_for_backward(gs.mu, gs.scale, gs.quat, gs.alpha)
        return gp_render_slices(ctx, gs, z, H, W, sigma_z, axis, view=v)

    @staticmethod
    def backward(fctx, g):
        ctx, z, H, W, sigma_z, axis, scale_mod, v = fctx.meta
        mu, scale, quat, alpha = fctx.saved_tensors
        gs = GaussianSet(mu, scale, quat, alpha, scale_mod)
        dm, ds, dq, da = gp_render_backward(ctx, gs, z, H, W, sigma_z, g.contiguous(), axis, view=v)
        return None, None, None, None, None, None, None, None, dm, ds, dq, da


def render(ctx, mu, scale, quat, alpha, z, H, W, sigma_z, axis=2, scale_mod=1.0, view=None):
    """Autograd-aware slice stack [S, H, W]; view = (R, t) for an oblique stack."""
    return SliceRender.apply(ctx, z, H, W, sigma_z, axis, scale_mod, view, mu, scale, quat, alpha)
