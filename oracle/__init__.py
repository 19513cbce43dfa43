"""FP64 CPU oracle of the GaussianPile slice projection operator (arXiv 2603.20611).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2603_20611_b300``) never imports it and
shares no code with it: the arithmetic lives in ``oracle.c`` (plain C, double
precision, OpenMP), built here with gcc into ``liboracle.so`` and called through
ctypes.

Functions follow the paper's route (Eq. 6-10 forward, Sec. S2 chain for the
backward, Eq. 12 for the voxelizer); see the header of ``oracle.c`` for the
conventions and the per-step citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, IEEE double)."""
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= newest_src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _View(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


def _view(view):
    """(R [3, 3], t [3]) -> the C view struct (kept alive by the caller)."""
    R, t = view
    R = _f64(R, (9,))
    t = _f64(t, (3,))
    return _View((ctypes.c_double * 9)(*R), (ctypes.c_double * 3)(*t))


class _Set(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("mu", ctypes.c_void_p),
                ("scale", ctypes.c_void_p),
                ("quat", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p),
                ("scale_mod", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        D = ctypes.c_double
        SP = ctypes.POINTER(_Set)
        VP = ctypes.POINTER(_View)
        lib.orc_render_view.argtypes = [SP, VP, I, P, I, I, D, P]
        lib.orc_render_points_view.argtypes = [SP, VP, I, P, D, I64, P, P, P, P]
        lib.orc_render_backward_view.argtypes = [SP, VP, I, P, I, I, D, P, P, P, P, P]
        lib.orc_count_evals_view.argtypes = [SP, VP, I, P, I, I, D, D]
        lib.orc_count_evals_view.restype = I64
        for f in ("orc_render_view", "orc_render_points_view", "orc_render_backward_view"):
            getattr(lib, f).restype = I
        lib.orc_render.argtypes = [SP, I, P, I, I, D, I, P]
        lib.orc_render_points.argtypes = [SP, I, P, D, I, I64, P, P, P, P]
        lib.orc_render_backward.argtypes = [SP, I, P, I, I, D, I, P, P, P, P, P]
        lib.orc_voxelize.argtypes = [SP, I, I, I, P]
        lib.orc_voxelize_points.argtypes = [SP, I64, P, P, P, P]
        lib.orc_voxelize_backward.argtypes = [SP, I, I, I, P, P, P, P, P]
        lib.orc_mse.argtypes = [I64, P, P, P]
        lib.orc_count_evals.argtypes = [SP, I, P, I, I, D, I, D]
        lib.orc_count_evals.restype = I64
        lib.orc_mse.restype = D
        lib.orc_num_threads.restype = I
        for f in ("orc_render", "orc_render_points", "orc_render_backward",
                  "orc_voxelize", "orc_voxelize_points", "orc_voxelize_backward"):
            getattr(lib, f).restype = I
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _GaussianSet:
    """Keeps fp64 copies alive while the C code reads them."""

    def __init__(self, mu, scale, quat, alpha, scale_mod=1.0):
        self.mu = _f64(mu, (-1, 3))
        self.scale = _f64(scale, (-1, 3))
        self.quat = _f64(quat, (-1, 4))
        self.alpha = _f64(alpha, (-1,))
        n = self.alpha.shape[0]
        assert self.mu.shape[0] == n and self.scale.shape[0] == n and self.quat.shape[0] == n
        self.n = n
        self.c = _Set(n, _ptr(self.mu).value, _ptr(self.scale).value,
                      _ptr(self.quat).value, _ptr(self.alpha).value, float(scale_mod))


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name} rejected its arguments (status {rc})")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def render(mu, scale, quat, alpha, z, H, W, sigma_z, axis=2, scale_mod=1.0, view=None):
    """Slice stack [S, H, W] by brute force over every Gaussian (Eq. 6-10).
    view = (R [3, 3], t [3]) selects a general slice orientation (axis is then
    ignored): camera coordinates x_c = R x + t, slice s is the plane z_c = z[s]."""
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    z = _f64(z, (-1,))
    out = np.zeros((z.shape[0], H, W), np.float64)
    if view is not None:
        v = _view(view)
        _check(_load().orc_render_view(ctypes.byref(g.c), ctypes.byref(v), z.shape[0], _ptr(z), H, W,
                                       float(sigma_z), _ptr(out)), "orc_render_view")
        return out
    _check(_load().orc_render(ctypes.byref(g.c), z.shape[0], _ptr(z), H, W,
                              float(sigma_z), axis, _ptr(out)), "orc_render")
    return out


def render_points(mu, scale, quat, alpha, z, sigma_z, pt_slice, pt_x, pt_y, axis=2,
                  scale_mod=1.0, view=None):
    """Eq. 10 at sample points (slice index, camera x, camera y)."""
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    z = _f64(z, (-1,))
    ps = np.ascontiguousarray(np.asarray(pt_slice, dtype=np.int32).reshape(-1))
    px = _f64(pt_x, (-1,))
    py = _f64(pt_y, (-1,))
    out = np.zeros(ps.shape[0], np.float64)
    if view is not None:
        v = _view(view)
        _check(_load().orc_render_points_view(ctypes.byref(g.c), ctypes.byref(v), z.shape[0], _ptr(z),
                                              float(sigma_z), ps.shape[0], _ptr(ps), _ptr(px), _ptr(py),
                                              _ptr(out)), "orc_render_points_view")
        return out
    _check(_load().orc_render_points(ctypes.byref(g.c), z.shape[0], _ptr(z), float(sigma_z),
                                     axis, ps.shape[0], _ptr(ps), _ptr(px), _ptr(py),
                                     _ptr(out)), "orc_render_points")
    return out


def render_backward(mu, scale, quat, alpha, z, H, W, sigma_z, dL_dI, axis=2, scale_mod=1.0, view=None):
    """(dL/dmu [n,3], dL/dscale [n,3], dL/dquat [n,4], dL/dalpha [n]) for a given dL/dI."""
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    z = _f64(z, (-1,))
    G = _f64(dL_dI, (z.shape[0], H, W))
    n = g.n
    dmu = np.zeros((n, 3)); ds = np.zeros((n, 3)); dq = np.zeros((n, 4)); da = np.zeros(n)
    if view is not None:
        v = _view(view)
        _check(_load().orc_render_backward_view(ctypes.byref(g.c), ctypes.byref(v), z.shape[0], _ptr(z), H,
                                                W, float(sigma_z), _ptr(G), _ptr(dmu), _ptr(ds),
                                                _ptr(dq), _ptr(da)), "orc_render_backward_view")
        return dmu, ds, dq, da
    _check(_load().orc_render_backward(ctypes.byref(g.c), z.shape[0], _ptr(z), H, W,
                                       float(sigma_z), axis, _ptr(G), _ptr(dmu), _ptr(ds),
                                       _ptr(dq), _ptr(da)), "orc_render_backward")
    return dmu, ds, dq, da


def voxelize(mu, scale, quat, alpha, X, Y, Z, scale_mod=1.0):
    """Volume [Z, Y, X] of Eq. 12 by brute force."""
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    out = np.zeros((Z, Y, X), np.float64)
    _check(_load().orc_voxelize(ctypes.byref(g.c), X, Y, Z, _ptr(out)), "orc_voxelize")
    return out


def voxelize_points(mu, scale, quat, alpha, px, py, pz, scale_mod=1.0):
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    px = _f64(px, (-1,)); py = _f64(py, (-1,)); pz = _f64(pz, (-1,))
    out = np.zeros(px.shape[0], np.float64)
    _check(_load().orc_voxelize_points(ctypes.byref(g.c), px.shape[0], _ptr(px), _ptr(py),
                                       _ptr(pz), _ptr(out)), "orc_voxelize_points")
    return out


def voxelize_backward(mu, scale, quat, alpha, X, Y, Z, dL_dV, scale_mod=1.0):
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    G = _f64(dL_dV, (Z, Y, X))
    n = g.n
    dmu = np.zeros((n, 3)); ds = np.zeros((n, 3)); dq = np.zeros((n, 4)); da = np.zeros(n)
    _check(_load().orc_voxelize_backward(ctypes.byref(g.c), X, Y, Z, _ptr(G), _ptr(dmu),
                                         _ptr(ds), _ptr(dq), _ptr(da)),
           "orc_voxelize_backward")
    return dmu, ds, dq, da


def count_evals(mu, scale, quat, alpha, z, H, W, sigma_z, axis=2, eps=1e-6, scale_mod=1.0, view=None):
    """Algorithmic evaluations of a render with culling bound eps (see oracle.h)."""
    g = _GaussianSet(mu, scale, quat, alpha, scale_mod)
    z = _f64(z, (-1,))
    if view is not None:
        v = _view(view)
        r = _load().orc_count_evals_view(ctypes.byref(g.c), ctypes.byref(v), z.shape[0], _ptr(z), H, W,
                                         float(sigma_z), float(eps))
        if r < 0:
            raise ValueError("orc_count_evals_view rejected its arguments")
        return int(r)
    r = _load().orc_count_evals(ctypes.byref(g.c), z.shape[0], _ptr(z), H, W, float(sigma_z), axis,
                                float(eps))
    if r < 0:
        raise ValueError("orc_count_evals rejected its arguments")
    return int(r)


def mse(I, T):
    """(L, dL/dI) of the mean squared error."""
    I = _f64(I); T = _f64(T, I.shape)
    g = np.zeros_like(I)
    L = _load().orc_mse(I.size, _ptr(I), _ptr(T), _ptr(g))
    return float(L), g


def count_vox_evals(mu, scale, quat, alpha, X, Y, Z, eps=1e-6, scale_mod=1.0):
    """Voxel centres inside each Gaussian's culling ellipsoid (x - mu)^T Sigma^-1
    (x - mu) <= 2 ln(1/eps) within the X x Y x Z grid: the algorithmic work of
    Eq. 12 under that culling (FP64 brute force over each bounding box)."""
    mu = np.asarray(mu, np.float64).reshape(-1, 3)
    sc = np.asarray(scale, np.float64).reshape(-1, 3) * scale_mod
    q = np.asarray(quat, np.float64).reshape(-1, 4)
    k2 = 2.0 * np.log(1.0 / eps)
    total = 0
    for i in range(mu.shape[0]):
        w, x, y, z = q[i] / np.linalg.norm(q[i])
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        S = R @ np.diag(sc[i] ** 2) @ R.T
        K = np.linalg.inv(S)
        h = np.sqrt(k2 * np.diag(S))
        lo = np.maximum(np.ceil(mu[i] - h - 0.5), 0).astype(int)
        hi = np.minimum(np.floor(mu[i] + h - 0.5), np.array([X, Y, Z]) - 1).astype(int)
        if np.any(hi < lo):
            continue
        g = np.stack(np.meshgrid(*[np.arange(lo[a], hi[a] + 1) + 0.5 for a in range(3)], indexing="ij"), -1)
        d = g - mu[i]
        total += int((np.einsum("...i,ij,...j->...", d, K, d) <= k2).sum())
    return total
