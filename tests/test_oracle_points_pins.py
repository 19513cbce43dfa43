"""Pins of the oracle's sampled-point renderer (Eq. 10 at arbitrary points).

``oracle.render_points`` (axis slices) and its ``view=`` form (oblique planes)
are the checkers behind every full-size parity test, so their own indexing is
pinned here, independently of the GPU path:

* at every pixel centre they equal the full-image renderer (itself pinned by
  closed forms, limits and quadrature in ``test_oracle_pins.py``), on all
  three slice axes and on an oblique view;
* at off-grid points they equal closed forms written out in numpy: the
  axis-aligned anisotropic Gaussian (P2) on each slice axis with the camera
  axes (y, z, x), (x, z, y), (x, y, z) of axes 0, 1, 2 (Sec. S1, R_c a
  permutation); the isotropic Gaussian (P1) under a general rotation (the
  covariance of an isotropic Gaussian does not change with R_c); and an
  anisotropic Gaussian under an oblique view through the conditional Gaussian
  of Sigma_c + sigma_z^2 e3 e3^T on the plane (Eq. 6-9 in closed form);
* points given in shuffled slice order, with several slices interleaved, land
  on the plane their slice index names.

A swapped x/y, a dropped pixel-centre offset or a wrong slice-index-to-plane
mapping fails one of these.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_20611_b300 import synth

# camera axes of the three slice axes: (in-plane x, in-plane y, slice normal)
CAMERA_AXES = {0: (1, 2, 0), 1: (0, 2, 1), 2: (0, 1, 2)}


def one(mu, scale, quat, alpha):
    return (np.array([mu], np.float64), np.array([scale], np.float64),
            np.array([quat], np.float64), np.array([alpha], np.float64))


def rot_wxyz(q):
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def small_set(seed, n, extent):
    g = synth.small(seed=seed, n=n, extent=extent)
    return (g.mu.astype(np.float64), g.scale.astype(np.float64), g.quat.astype(np.float64),
            g.alpha.astype(np.float64))


def pixel_centres(S, H, W):
    s, iy, ix = np.meshgrid(np.arange(S), np.arange(H), np.arange(W), indexing="ij")
    return s.ravel(), ix.ravel() + 0.5, iy.ravel() + 0.5


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_points_at_pixel_centres_equal_render(axis):
    g = small_set(31 + axis, 60, (20, 18, 16))
    ext = (20, 18, 16)
    px_ax, py_ax, _ = CAMERA_AXES[axis]
    H, W = ext[py_ax], ext[px_ax]
    z = np.array([0.5, 3.25, 7.5, 11.0, 15.5])
    img = oracle.render(*g, z, H, W, 2.0, axis=axis)
    s, x, y = pixel_centres(len(z), H, W)
    pts = oracle.render_points(*g, z, 2.0, s, x, y, axis=axis)
    ref = img.reshape(-1)
    assert np.abs(pts - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.linalg.norm(pts - ref) <= 1e-13 * np.linalg.norm(ref)


def test_view_points_at_pixel_centres_equal_render():
    g = small_set(41, 60, (24, 24, 24))
    R = Rotation.random(random_state=5).as_matrix()
    t = np.array([12.0, 12.0, 0.0]) - R @ np.array([12.0, 12.0, 12.0])
    z = np.array([-4.0, -0.5, 0.0, 2.5, 6.0])
    H, W = 22, 26
    img = oracle.render(*g, z, H, W, 3.0, view=(R, t))
    s, x, y = pixel_centres(len(z), H, W)
    pts = oracle.render_points(*g, z, 3.0, s, x, y, view=(R, t))
    ref = img.reshape(-1)
    assert np.abs(pts - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.linalg.norm(pts - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_off_grid_axis_aligned_closed_form(axis):
    """P2 on each slice axis at points off the pixel grid."""
    mu, sc, alpha, sig = np.array([8.3, 6.9, 5.2]), np.array([1.3, 2.4, 3.1]), 0.7, 1.5
    z = np.array([2.0, 4.75, 9.5])
    pts = np.array([[0, 3.37, 11.81], [1, 7.02, 4.44], [2, 9.9, 0.13], [1, 12.6, 8.08], [0, 5.0, 5.0]])
    got = oracle.render_points(*one(mu, sc, (1, 0, 0, 0), alpha), z, sig, pts[:, 0], pts[:, 1], pts[:, 2],
                               axis=axis)
    ax, ay, an = CAMERA_AXES[axis]
    for k, (s, x, y) in enumerate(pts):
        d = mu[an] - z[int(s)]
        ref = alpha / (sc[ax] * sc[ay]) * math.exp(-0.5 * d * d / (sc[an] ** 2 + sig * sig)) \
            * math.exp(-0.5 * ((x - mu[ax]) ** 2 / sc[ax] ** 2 + (y - mu[ay]) ** 2 / sc[ay] ** 2))
        assert got[k] == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_off_grid_isotropic_closed_form_under_a_view():
    """P1 with a general camera rotation: Sigma_c = s^2 I for every R_c, so the
    response at camera point (x, y) on plane z_c is alpha/s^2 exp(-(mu_c,z -
    z_c)^2 / 2(s^2 + sigma_z^2)) exp(-|(x, y) - mu_c,xy|^2 / 2 s^2)."""
    mu, s, alpha, sig = np.array([9.2, 4.1, 7.7]), 1.9, 0.45, 2.5
    R = Rotation.random(random_state=11).as_matrix()
    t = np.array([3.0, -2.0, 1.5])
    muc = R @ mu + t
    z = np.array([muc[2] - 3.1, muc[2] + 0.4, muc[2] + 2.2])
    pts = np.array([[2, muc[0] + 0.37, muc[1] - 1.81], [0, muc[0] - 2.2, muc[1] + 0.6],
                    [1, muc[0] + 3.37, muc[1] + 1.81], [2, muc[0], muc[1]]])
    got = oracle.render_points(*one(mu, (s, s, s), (0.3, 0.5, -0.1, 0.8), alpha), z, sig,
                               pts[:, 0], pts[:, 1], pts[:, 2], view=(R, t))
    for k, (si, x, y) in enumerate(pts):
        d = muc[2] - z[int(si)]
        ref = alpha / s ** 2 * math.exp(-0.5 * d * d / (s * s + sig * sig)) \
            * math.exp(-0.5 * ((x - muc[0]) ** 2 + (y - muc[1]) ** 2) / s ** 2)
        assert got[k] == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_off_grid_anisotropic_conditional_form_under_a_view():
    """An anisotropic Gaussian under an oblique view: Eq. 6-9 in closed form.
    With Sigma_c = R Sigma R^T and v = Sigma_c,zz + sigma_z^2, the plane sees
    mean mu_c,xy - Sigma_c,xz (mu_c,z - z) / v, covariance Sigma_c,xy -
    Sigma_c,xz Sigma_c,zx / v and amplitude alpha exp(-(mu_c,z - z)^2 / 2v) /
    sqrt(det)."""
    mu, sc, q, alpha, sig = np.array([5.0, 6.0, 7.0]), np.array([1.2, 2.6, 0.9]), (0.7, 0.2, -0.4, 0.5), 0.9, 1.7
    Rw = rot_wxyz(np.array(q) / np.linalg.norm(q))
    Sig = Rw @ np.diag(sc ** 2) @ Rw.T
    R = Rotation.random(random_state=23).as_matrix()
    t = np.array([10.0, 9.0, -4.0])
    muc = R @ mu + t
    Sc = R @ Sig @ R.T
    z = np.array([muc[2] + 1.3, muc[2] - 0.6])
    rng = np.random.default_rng(3)
    pts = np.column_stack([rng.integers(0, 2, 12), muc[0] + rng.uniform(-3, 3, 12),
                           muc[1] + rng.uniform(-3, 3, 12)])
    got = oracle.render_points(*one(mu, sc, q, alpha), z, sig, pts[:, 0], pts[:, 1], pts[:, 2], view=(R, t))
    v = Sc[2, 2] + sig * sig
    S2 = Sc[:2, :2] - np.outer(Sc[:2, 2], Sc[2, :2]) / v
    Ci = np.linalg.inv(S2)
    for k, (si, x, y) in enumerate(pts):
        d = muc[2] - z[int(si)]
        m2 = muc[:2] - Sc[:2, 2] * d / v
        dd = np.array([x, y]) - m2
        ref = alpha * math.exp(-0.5 * d * d / v) / math.sqrt(np.linalg.det(S2)) * math.exp(-0.5 * dd @ Ci @ dd)
        assert got[k] == pytest.approx(ref, rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("axis", [1, 2])
def test_shuffled_slice_order(axis):
    """Points of five planes given interleaved and in random order: each one
    takes the value of its own plane's image at that pixel."""
    g = small_set(51, 40, (16, 16, 16))
    z = np.array([1.5, 4.5, 8.0, 12.5, 14.0])
    img = oracle.render(*g, z, 16, 16, 2.0, axis=axis)
    rng = np.random.default_rng(9)
    s = rng.permutation(np.repeat(np.arange(5), 30))
    ix = rng.integers(0, 16, s.size)
    iy = rng.integers(0, 16, s.size)
    got = oracle.render_points(*g, z, 2.0, s, ix + 0.5, iy + 0.5, axis=axis)
    ref = img[s, iy, ix]
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(img).max())
    # the same points one plane at a time
    for k in range(5):
        sel = s == k
        one_plane = oracle.render_points(*g, z[k:k + 1], 2.0, np.zeros(sel.sum(), np.int32), ix[sel] + 0.5,
                                         iy[sel] + 0.5, axis=axis)
        np.testing.assert_allclose(one_plane, got[sel], rtol=1e-13, atol=1e-300)


def test_points_validate_slice_indices():
    g = small_set(61, 5, (8, 8, 8))
    z = np.array([0.5, 1.5])
    for bad in (-1, 2):
        with pytest.raises(ValueError):
            oracle.render_points(*g, z, 2.0, [0, bad], [1.5, 2.5], [1.5, 2.5])
    assert oracle.render_points(*g, z, 2.0, [], [], []).shape == (0,)
