"""What the device's culling may leave out, per pixel and per parameter.

The device drops a (Gaussian, plane) pair whose axial factor opacity_r is
below eps, and inside a kept pair every pixel whose in-plane Mahalanobis
distance m = d^T Sigma_2d^-1 d exceeds k^2 = 2 ln(1/eps) (Sec. 4.2 leaves the
threshold open; eps = 1e-6 is this library's reading).  It may evaluate more
pixels than that (whole culling cells), never fewer.  Every term
f = a~ exp(-m/2) is >= 0, so per pixel

    0 <= I_oracle - I_device <= b(p) = sum over pairs of f [opacity_r < eps or m > k^2]

and the gradient of parameter theta of Gaussian i differs by at most
sum over its culled (plane, pixel) terms of |dL/dI| * f * |d ln f / d theta|.

Both are computed here in float64 numpy from the closed form of Eq. 6-9
(Sigma_c = R_c Sigma R_c^T, v = Sigma_c,zz + sigma_z^2, Sigma_2d = Sigma_c,xy -
Sigma_c,xz Sigma_c,zx / v, mu_2d = mu_c,xy - Sigma_c,xz delta / v, a~ = alpha
exp(-delta^2 / 2v) / sqrt(det Sigma_2d)); d ln f / d theta by central
differences of ln f, which is smooth where f itself underflows.  This is a
tolerance, not a checker: ``tests/test_truncation_bound.py`` pins the closed
form to the oracle.  No arithmetic here is shared with the device path or the
oracle.
"""
import math

import numpy as np
from scipy.spatial.transform import Rotation

EPS = 1e-6
# camera rows of the three slice axes (in-plane x, in-plane y, slice normal)
AXIS_ROWS = {0: (1, 2, 0), 1: (0, 2, 1), 2: (0, 1, 2)}


def axis_view(axis):
    R = np.zeros((3, 3))
    for r, c in enumerate(AXIS_ROWS[axis]):
        R[r, c] = 1.0
    return R, np.zeros(3)


def _pair_params(mu, scale, quat, alpha, z, sigma, mod, R, t):
    """ln a~ [S, n], mu_2d [S, n, 2], C = Sigma_2d^-1 [n, 2, 2], opacity_r [S, n]."""
    q = quat / np.linalg.norm(quat, axis=-1, keepdims=True)
    Rw = Rotation.from_quat(np.stack([q[..., 1], q[..., 2], q[..., 3], q[..., 0]], -1)).as_matrix()
    s = mod * scale
    Sig = np.einsum('nij,nj,nkj->nik', Rw, s * s, Rw)
    Sc = np.einsum('ij,njk,lk->nil', R, Sig, R)
    muc = mu @ R.T + t
    v = Sc[:, 2, 2] + sigma * sigma
    b = Sc[:, :2, 2]
    S2 = Sc[:, :2, :2] - np.einsum('ni,nj->nij', b, b) / v[:, None, None]
    det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
    C = np.stack([np.stack([S2[:, 1, 1], -S2[:, 0, 1]], -1), np.stack([-S2[:, 1, 0], S2[:, 0, 0]], -1)], -2)
    C = C / det[:, None, None]
    delta = muc[None, :, 2] - z[:, None]
    ln_op = -0.5 * delta * delta / v[None, :]
    with np.errstate(divide="ignore"):
        ln_at = np.log(alpha)[None, :] + ln_op - 0.5 * np.log(det)[None, :]
    mu2 = muc[None, :, :2] - b[None, :, :] * (delta / v[None, :])[..., None]
    return ln_at, mu2, C, np.exp(ln_op)


def _maha(mu2, C, px, py):
    """m [S, n, P] for pixel centres (px, py) [P]."""
    dx = px[None, None, :] - mu2[..., 0:1]
    dy = py[None, None, :] - mu2[..., 1:2]
    return dx * (C[None, :, 0, 0, None] * dx + C[None, :, 0, 1, None] * dy) + \
        dy * (C[None, :, 1, 0, None] * dx + C[None, :, 1, 1, None] * dy)


def _as64(g):
    return (np.asarray(g.mu, np.float64).reshape(-1, 3), np.asarray(g.scale, np.float64).reshape(-1, 3),
            np.asarray(g.quat, np.float64).reshape(-1, 4), np.asarray(g.alpha, np.float64).reshape(-1))


def render_closed_form(g, z, H, W, sigma, mod=1.0, view=None, chunk=64):
    """[S, H, W]: every term, no culling (pinned against the oracle's render)."""
    return _terms(g, z, H, W, sigma, mod, view, chunk, culled_only=False)


def forward_bound(g, z, H, W, sigma, mod=1.0, view=None, chunk=64, eps=EPS):
    """b [S, H, W]: the sum of the terms the device's culling may drop."""
    return _terms(g, z, H, W, sigma, mod, view, chunk, culled_only=True, eps=eps)


def _terms(g, z, H, W, sigma, mod, view, chunk, culled_only, eps=EPS):
    mu, sc, qu, al = _as64(g)
    z = np.asarray(z, np.float64).reshape(-1)
    R, t = (np.asarray(view[0], np.float64), np.asarray(view[1], np.float64)) if view is not None else axis_view(2)
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    px, py = xx.ravel(), yy.ravel()
    out = np.zeros((z.size, H * W))
    for a in range(0, al.size, chunk):
        sl = slice(a, a + chunk)
        ln_at, mu2, C, op = _pair_params(mu[sl], sc[sl], qu[sl], al[sl], z, sigma, mod, R, t)
        m = _maha(mu2, C, px, py)
        f = np.exp(ln_at[..., None] - 0.5 * m)
        if culled_only:
            f = np.where((op[..., None] < eps) | (m > 2.0 * math.log(1.0 / eps)), f, 0.0)
        out += f.sum(axis=1)
    return out.reshape(z.size, H, W)


def gradient_bound(g, z, H, W, sigma, G, mod=1.0, view=None, chunk=32, h_rel=1e-6, eps=EPS):
    """Per-parameter bounds (mu [n,3], scale [n,3], quat [n,4], alpha [n]) on
    |dL/dtheta(oracle) - dL/dtheta(device)| for the per-pixel weights G = dL/dI."""
    mu, sc, qu, al = _as64(g)
    z = np.asarray(z, np.float64).reshape(-1)
    R, t = (np.asarray(view[0], np.float64), np.asarray(view[1], np.float64)) if view is not None else axis_view(2)
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    px, py = xx.ravel(), yy.ravel()
    aG = np.abs(np.asarray(G, np.float64)).reshape(z.size, 1, H * W)
    n = al.size
    bmu, bsc, bqu, bal = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n)
    for a in range(0, n, chunk):
        sl = slice(a, a + chunk)
        p0 = [mu[sl], sc[sl], qu[sl], al[sl]]
        ln_at, mu2, C, op = _pair_params(*p0, z, sigma, mod, R, t)
        m = _maha(mu2, C, px, py)
        w = aG * np.where((op[..., None] < eps) | (m > 2.0 * math.log(1.0 / eps)),
                          np.exp(ln_at[..., None] - 0.5 * m), 0.0)
        # alpha enters ln f as ln alpha
        with np.errstate(divide="ignore", invalid="ignore"):
            bal[sl] = np.where(p0[3] > 0, w.sum(axis=(0, 2)) / p0[3], 0.0)
        for grp, (arr, out) in enumerate(((mu, bmu), (sc, bsc), (qu, bqu))):
            for j in range(arr.shape[1]):
                h = h_rel * np.maximum(np.abs(arr[sl, j]), 1.0)
                lnf = []
                for sgn in (1.0, -1.0):
                    p = [x.copy() for x in p0]
                    p[grp][:, j] += sgn * h
                    la, m2, Cc, _ = _pair_params(*p, z, sigma, mod, R, t)
                    lnf.append(la[..., None] - 0.5 * _maha(m2, Cc, px, py))
                with np.errstate(invalid="ignore"):
                    dlnf = (lnf[0] - lnf[1]) / (2.0 * h)[None, :, None]
                out[sl, j] = np.where(w > 0, w * np.abs(dlnf), 0.0).sum(axis=(0, 2))
    # central differences are exact for the quadratic parts and O(h^2) elsewhere
    return tuple(1.01 * b for b in (bmu, bsc, bqu, bal))
