"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own route (inverse-covariance update,
Eq. 6-9).  Each compares it with something independent of it:

* closed forms of a single isotropic / axis-aligned Gaussian;
* the two limits drawn in Fig. 1(b) (sigma_z -> inf, all-in-focus marginal) and
  Fig. 1(c) (sigma_z -> 0, the 3-D Gaussian restricted to the plane);
* adaptive quadrature of the convolution integral Eq. 5 (Sec. 4.2 / Sec. S1),
  which equals the paper's Eq. 9 response times the known factor
  F = sqrt(2 pi) sigma_z sqrt(det Sigma / (Sigma_zz + sigma_z^2));
* mass: a slice integrates to 2 pi alpha opacity_r (Eq. 9 "preserving total
  energy"), a stack to (2 pi)^(3/2) alpha sqrt(Sigma_zz + sigma_z^2), a volume
  to (2 pi)^(3/2) alpha sqrt(det Sigma) (Eq. 12);
* linearity (Sec. S1, "linearity of the imaging model"), integer-shift and
  90-degree-rotation equivariance;
* central finite differences of every gradient (Sec. 4.3 / S2), and the exact
  relations dI/da~ = exp(.) (Eq. 10) and dL/dalpha = dL/da~ opacity_r /
  sqrt(det Sigma_2d) (Sec. 4.3).

Rotations in the tests come from scipy (scalar-last quaternions), covariances
and inverses from numpy, integrals from scipy.integrate.quad.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_20611_b300 import synth

TWO_PI = 2.0 * math.pi


def rot(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def cov(scale, q_wxyz, mod=1.0):
    R = rot(q_wxyz)
    S = np.diag(mod * np.asarray(scale, np.float64))
    return R @ S @ S @ R.T


def one(mu, scale, quat, alpha):
    return (np.array([mu], np.float64), np.array([scale], np.float64),
            np.array([quat], np.float64), np.array([alpha], np.float64))


def pixel_grid(H, W):
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    return xx, yy


RNG = np.random.Generator(np.random.PCG64(7))
Q_RAND = RNG.standard_normal(4)
Q_RAND /= np.linalg.norm(Q_RAND)


# --------------------------------------------------------------- closed forms

def test_isotropic_closed_form():
    """P1: Sigma = s^2 I gives Sigma_2d = s^2 I_2, mu_2d = mu_xy and
    I = alpha / s^2 exp(-delta^2 / 2(s^2 + sigma_z^2)) exp(-|p - mu_xy|^2 / 2 s^2)."""
    mu, s, alpha, sig = (7.3, 9.1, 4.2), 1.7, 0.8, 2.0
    z = np.array([0.5, 2.5, 4.5, 7.5])
    H, W = 16, 18
    I = oracle.render(*one(mu, (s, s, s), Q_RAND, alpha), z, H, W, sig)
    xx, yy = pixel_grid(H, W)
    for k, zs in enumerate(z):
        d2 = (xx - mu[0]) ** 2 + (yy - mu[1]) ** 2
        ref = alpha / s ** 2 * math.exp(-0.5 * (mu[2] - zs) ** 2 / (s * s + sig * sig)) \
            * np.exp(-0.5 * d2 / s ** 2)
        np.testing.assert_allclose(I[k], ref, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("quat,swap", [((1, 0, 0, 0), False),
                                       ((math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)), True)])
def test_axis_aligned_closed_form(quat, swap):
    """P2: R = I (or a quarter turn about z, which swaps s_x and s_y):
    I = alpha/(s_x s_y) exp(-delta^2/2(s_z^2+sigma_z^2)) exp(-dx^2/2s_x^2 - dy^2/2s_y^2)."""
    mu, sc, alpha, sig = (8.0, 6.5, 3.0), (1.3, 2.4, 3.1), 0.6, 1.5
    z = np.array([1.5, 3.0, 6.0])
    H, W = 14, 16
    I = oracle.render(*one(mu, sc, quat, alpha), z, H, W, sig)
    sx, sy, sz = sc
    if swap:
        sx, sy = sy, sx
    xx, yy = pixel_grid(H, W)
    for k, zs in enumerate(z):
        ref = alpha / (sx * sy) * math.exp(-0.5 * (mu[2] - zs) ** 2 / (sz * sz + sig * sig)) \
            * np.exp(-0.5 * ((xx - mu[0]) ** 2 / sx ** 2 + (yy - mu[1]) ** 2 / sy ** 2))
        np.testing.assert_allclose(I[k], ref, rtol=1e-11, atol=1e-300)


# -------------------------------------------------------------------- limits

def test_all_in_focus_limit():
    """P3, Fig. 1(b): sigma_z -> inf leaves the xy marginal of the 3-D Gaussian,
    I = alpha / sqrt(det Sigma_xy) exp(-1/2 d^T Sigma_xy^-1 d), the same on every slice."""
    mu, sc, alpha = (9.0, 8.0, 5.0), (1.2, 2.5, 1.8), 0.9
    Sig = cov(sc, Q_RAND)
    Sxy = Sig[:2, :2]
    Ki = np.linalg.inv(Sxy)
    H, W = 18, 18
    z = np.array([0.5, 5.0, 40.0])
    I = oracle.render(*one(mu, sc, Q_RAND, alpha), z, H, W, 1e6)
    xx, yy = pixel_grid(H, W)
    dx, dy = xx - mu[0], yy - mu[1]
    m = Ki[0, 0] * dx * dx + 2 * Ki[0, 1] * dx * dy + Ki[1, 1] * dy * dy
    ref = alpha / math.sqrt(np.linalg.det(Sxy)) * np.exp(-0.5 * m)
    for k in range(len(z)):
        np.testing.assert_allclose(I[k], ref, rtol=1e-8, atol=1e-14)


def test_zero_thickness_limit():
    """P4, Fig. 1(c): sigma_z -> 0 leaves the 3-D Gaussian on the plane, scaled by
    1/sqrt(det Sigma_cond) with det Sigma_cond = det Sigma / Sigma_zz (Schur)."""
    mu, sc, alpha = (8.2, 7.7, 6.1), (1.4, 2.2, 1.9), 0.7
    Sig = cov(sc, Q_RAND)
    K = np.linalg.inv(Sig)
    det_cond = np.linalg.det(Sig) / Sig[2, 2]
    H, W = 16, 16
    z = np.array([4.5, 6.0, 7.5])
    I = oracle.render(*one(mu, sc, Q_RAND, alpha), z, H, W, 1e-4)
    xx, yy = pixel_grid(H, W)
    for k, zs in enumerate(z):
        d = np.stack([xx - mu[0], yy - mu[1], np.full_like(xx, zs - mu[2])], -1)
        m = np.einsum("...i,ij,...j->...", d, K, d)
        ref = alpha * np.exp(-0.5 * m) / math.sqrt(det_cond)
        np.testing.assert_allclose(I[k], ref, rtol=1e-6, atol=1e-12)
        # the same through the voxelizer (Eq. 12) at the plane
        v = oracle.voxelize_points(*one(mu, sc, Q_RAND, alpha), xx.ravel(), yy.ravel(),
                                   np.full(xx.size, zs))
        np.testing.assert_allclose(I[k].ravel() * math.sqrt(det_cond), v, rtol=1e-6, atol=1e-12)


# ------------------------------------------------------- Eq. 5 by quadrature

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_convolution_integral_quadrature(axis):
    """P5: integral of h(t) g(x, y, t) dt (Eq. 5) by adaptive quadrature equals the
    Eq. 9/10 response times F = sqrt(2 pi) sigma_z sqrt(det Sigma / (Sigma_cc + sigma_z^2)),
    for a rotated anisotropic Gaussian on slices through each of the three axes.
    Camera frames: axis 2 (x,y,z), axis 1 (x,z,y), axis 0 (y,z,x)."""
    perm = {2: (0, 1, 2), 1: (0, 2, 1), 0: (1, 2, 0)}[axis]
    mu = np.array([6.4, 7.1, 5.3])
    sc = (1.1, 2.6, 1.7)
    alpha, sig = 0.75, 1.3
    Sig = cov(sc, Q_RAND)
    K = np.linalg.inv(Sig)
    Pm = np.zeros((3, 3))
    for j in range(3):
        Pm[j, perm[j]] = 1.0
    Sc = Pm @ Sig @ Pm.T
    F = math.sqrt(TWO_PI) * sig * math.sqrt(np.linalg.det(Sig) / (Sc[2, 2] + sig * sig))
    z = np.array([3.5, 5.0, 8.25])
    H, W = 12, 12
    I = oracle.render(*one(mu, sc, Q_RAND, alpha), z, H, W, sig, axis=axis)
    pts = [(1, 2), (5, 6), (7, 4), (10, 9), (3, 11)]
    for k, zs in enumerate(z):
        for (iy, ix) in pts:
            xc, yc = ix + 0.5, iy + 0.5

            def integrand(t):
                xcam = np.array([xc, yc, zs + t])  # camera-frame point, world = P^T xcam
                d = Pm.T @ xcam - mu
                return math.exp(-t * t / (2 * sig * sig)) * alpha * math.exp(-0.5 * d @ K @ d)

            val, err = integrate.quad(integrand, -60, 60, epsabs=1e-15, epsrel=1e-12, limit=200)
            assert I[k, iy, ix] * F == pytest.approx(val, rel=1e-9, abs=1e-16)


# ---------------------------------------------------------------------- mass

def test_slice_mass():
    """P6: a slice sums to 2 pi alpha opacity_r with opacity_r = exp(-delta^2/2v),
    v = Sigma_zz + sigma_z^2 (grid sums of a Gaussian with std >= 1 px are exact
    to far below 1e-8 by Poisson summation)."""
    mu, sc, alpha, sig = (24.3, 23.8, 12.0), (1.5, 3.0, 2.0), 0.6, 2.0
    Sig = cov(sc, Q_RAND)
    v = Sig[2, 2] + sig * sig
    z = np.array([9.5, 12.0, 15.5])
    I = oracle.render(*one(mu, sc, Q_RAND, alpha), z, 48, 48, sig)
    for k, zs in enumerate(z):
        ref = TWO_PI * alpha * math.exp(-0.5 * (mu[2] - zs) ** 2 / v)
        assert I[k].sum() == pytest.approx(ref, rel=1e-9)


def test_stack_mass_conservation():
    """P6: over slices one voxel apart, sum_s sum_p I_s = (2 pi)^(3/2) sum_i alpha_i
    sqrt(Sigma_zz,i + sigma_z^2) (mass conservation: the slice sums times the
    slice spacing give the total integrated intensity, in the paper's Eq. 9
    amplitude)."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 5
    mu = np.column_stack([rng.uniform(18, 30, n), rng.uniform(18, 30, n), rng.uniform(28, 36, n)])
    sc = rng.uniform(1.2, 2.5, (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    al = rng.uniform(0.2, 1.0, n)
    sig = 2.0
    z = np.arange(64) + 0.5
    I = oracle.render(mu, sc, q, al, z, 48, 48, sig)
    ref = sum((TWO_PI) ** 1.5 * al[i] * math.sqrt(cov(sc[i], q[i])[2, 2] + sig * sig)
              for i in range(n))
    assert I.sum() == pytest.approx(ref, rel=1e-8)


def test_voxel_mass():
    """P6 for Eq. 12: the volume sums to (2 pi)^(3/2) sum_i alpha_i sqrt(det Sigma_i)."""
    rng = np.random.Generator(np.random.PCG64(12))
    n = 4
    mu = rng.uniform(12, 20, (n, 3))
    sc = rng.uniform(1.1, 2.2, (n, 3))
    q = rng.standard_normal((n, 4))
    al = rng.uniform(0.2, 1.0, n)
    V = oracle.voxelize(mu, sc, q, al, 32, 32, 32)
    ref = sum(TWO_PI ** 1.5 * al[i] * math.sqrt(np.linalg.det(cov(sc[i], q[i] / np.linalg.norm(q[i]))))
              for i in range(n))
    assert V.sum() == pytest.approx(ref, rel=1e-8)


def test_voxel_closed_form_scale_mod():
    """Eq. 12 at single points against numpy, with the scale modifier of Sec. S1
    (S = diag(mod s))."""
    mu, sc, alpha, mod = (5.0, 6.0, 7.0), (1.0, 1.5, 2.0), 0.4, 1.3
    Sig = cov(sc, Q_RAND, mod)
    K = np.linalg.inv(Sig)
    pts = np.array([[5.5, 6.5, 7.5], [3.5, 8.5, 6.5], [7.5, 5.5, 9.5]])
    v = oracle.voxelize_points(*one(mu, sc, Q_RAND, alpha), pts[:, 0], pts[:, 1], pts[:, 2],
                               scale_mod=mod)
    ref = [alpha * math.exp(-0.5 * (p - mu) @ K @ (p - mu)) for p in pts]
    np.testing.assert_allclose(v, ref, rtol=1e-12)


# ------------------------------------------------------ structure of the sum

def test_linearity():
    """P7: I(G1 u G2) = I(G1) + I(G2) (Sec. S1, linearity of the imaging model)."""
    g = synth.small(seed=5, n=40, extent=(16, 16, 8))
    z = synth.slice_positions(range(8))
    a = oracle.render(g.mu[:25], g.scale[:25], g.quat[:25], g.alpha[:25], z, 16, 16, 2.0)
    b = oracle.render(g.mu[25:], g.scale[25:], g.quat[25:], g.alpha[25:], z, 16, 16, 2.0)
    ab = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 16, 16, 2.0)
    np.testing.assert_allclose(ab, a + b, rtol=1e-12, atol=1e-15)


def test_integer_shift_equivariance():
    """P8: shifting every mean by whole pixels shifts the image by the same pixels."""
    g = synth.small(seed=6, n=12, extent=(12, 12, 8))
    mu = g.mu.astype(np.float64) + np.array([10.0, 10.0, 0.0])
    z = synth.slice_positions([2, 5])
    a = oracle.render(mu, g.scale, g.quat, g.alpha, z, 40, 40, 1.5)
    b = oracle.render(mu + np.array([3.0, -2.0, 0.0]), g.scale, g.quat, g.alpha, z, 40, 40, 1.5)
    np.testing.assert_allclose(b[:, 12:30, 13:33], a[:, 14:32, 10:30], rtol=1e-10, atol=1e-15)


def test_quarter_turn_equivariance():
    """P8: rotating the set by 90 degrees about z (quaternion product, mean rotated
    about the image centre) rotates each slice image by 90 degrees."""
    g = synth.small(seed=8, n=15, extent=(20, 20, 8))
    c = 10.0
    qz = Rotation.from_euler("z", 90, degrees=True)
    mu = g.mu.astype(np.float64)
    mu2 = mu.copy()
    mu2[:, 0] = c - (mu[:, 1] - c)
    mu2[:, 1] = c + (mu[:, 0] - c)
    q = g.quat.astype(np.float64)
    r = qz * Rotation.from_quat(np.column_stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]]))
    qs = r.as_quat()
    q2 = np.column_stack([qs[:, 3], qs[:, 0], qs[:, 1], qs[:, 2]])
    z = synth.slice_positions([1, 4, 6])
    a = oracle.render(mu, g.scale, q, g.alpha, z, 20, 20, 2.0)
    b = oracle.render(mu2, g.scale, q2, g.alpha, z, 20, 20, 2.0)
    # pixel (ix, iy) of a lands on (ix', iy') = (2c - 1 - iy, ix) in b, i.e.
    # b[r, col] = a[2c - 1 - col, r]: a clockwise quarter turn of the array
    np.testing.assert_allclose(b, np.rot90(a, k=-1, axes=(1, 2)), rtol=1e-10, atol=1e-14)


def test_slice_axes_agree_with_transposed_volume():
    """P8: slicing along x (axis 0, camera (y, z, x)) equals slicing along z of the
    set whose coordinates are relabelled (x, y, z) <- (y, z, x)."""
    g = synth.small(seed=9, n=10, extent=(12, 12, 12))
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], np.float64)  # proper rotation
    rP = Rotation.from_matrix(P)
    q = g.quat.astype(np.float64)
    r = rP * Rotation.from_quat(np.column_stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]]))
    qs = r.as_quat()
    q2 = np.column_stack([qs[:, 3], qs[:, 0], qs[:, 1], qs[:, 2]])
    mu2 = g.mu.astype(np.float64) @ P.T
    z = synth.slice_positions([3, 7])
    a = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 12, 12, 1.7, axis=0)
    b = oracle.render(mu2, g.scale, q2, g.alpha, z, 12, 12, 1.7, axis=2)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-14)


def test_scale_mod_equals_scaled_scales():
    """Sec. S1: S = diag(mod s), so (s, mod) renders like (mod s, 1)."""
    g = synth.small(seed=10, n=8, extent=(12, 12, 6))
    z = synth.slice_positions([1, 3])
    a = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 12, 12, 1.0, scale_mod=1.4)
    b = oracle.render(g.mu, 1.4 * g.scale.astype(np.float64), g.quat, g.alpha, z, 12, 12, 1.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


def test_quaternion_scale_invariance():
    """Sec. S1: R comes from the unit quaternion, so q and 3.7 q render alike."""
    g = synth.small(seed=12, n=6, extent=(10, 10, 6))
    z = synth.slice_positions([2])
    a = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 10, 10, 1.0)
    b = oracle.render(g.mu, g.scale, 3.7 * g.quat.astype(np.float64), g.alpha, z, 10, 10, 1.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


def test_empty_set_and_empty_stack():
    z = synth.slice_positions([0, 1])
    e = np.zeros((0, 3))
    I = oracle.render(e, e, np.zeros((0, 4)), np.zeros(0), z, 4, 5, 1.0)
    assert I.shape == (2, 4, 5) and not I.any()
    I0 = oracle.render(*one((1, 1, 1), (1, 1, 1), (1, 0, 0, 0), 1.0), np.zeros(0), 4, 4, 1.0)
    assert I0.shape == (0, 4, 4)
    with pytest.raises(ValueError):
        oracle.render(*one((1, 1, 1), (1, 1, 1), (1, 0, 0, 0), 1.0), z, 4, 4, 0.0)


# ------------------------------------------------------------------ gradients

def _fd_check(fwd, params, grads, G, h_rel=1e-6, rtol=2e-6):
    """Central differences of L = sum G * fwd(params) against the analytic grads."""
    for name, arr in params.items():
        ana = grads[name]
        flat = arr.reshape(-1)
        num = np.zeros_like(flat)
        for k in range(flat.size):
            h = h_rel * max(1.0, abs(flat[k]))
            old = flat[k]
            flat[k] = old + h
            lp = float((G * fwd()).sum())
            flat[k] = old - h
            lm = float((G * fwd()).sum())
            flat[k] = old
            num[k] = (lp - lm) / (2 * h)
        scale = max(np.abs(num).max(), 1e-12)
        np.testing.assert_allclose(ana.reshape(-1), num, rtol=rtol, atol=rtol * scale,
                                   err_msg=f"gradient of {name}")


@pytest.mark.parametrize("axis,mod", [(2, 1.0), (0, 1.2), (1, 0.9)])
def test_render_gradient_finite_differences(axis, mod):
    """P9: analytic oracle gradient of all 11 parameters per Gaussian vs central
    differences in FP64, on a tiny stack (5 Gaussians, 14 x 12 x 4)."""
    rng = np.random.Generator(np.random.PCG64(100 + axis))
    n, H, W = 5, 12, 14
    mu = np.column_stack([rng.uniform(3, 11, n), rng.uniform(3, 9, n), rng.uniform(1, 5, n)])
    sc = rng.uniform(0.8, 2.2, (n, 3))
    q = rng.standard_normal((n, 4)) * 1.3
    al = rng.uniform(0.2, 1.0, n)
    z = np.array([1.0, 2.5, 3.25, 5.0])
    sig = 1.4
    G = rng.standard_normal((len(z), H, W))
    p = {"mu": mu, "scale": sc, "quat": q, "alpha": al}

    def fwd():
        return oracle.render(mu, sc, q, al, z, H, W, sig, axis=axis, scale_mod=mod)

    dmu, ds, dq, da = oracle.render_backward(mu, sc, q, al, z, H, W, sig, G, axis=axis,
                                             scale_mod=mod)
    _fd_check(fwd, p, {"mu": dmu, "scale": ds, "quat": dq, "alpha": da}, G)


def test_alpha_gradient_is_exact_relation():
    """Sec. 4.3: dL/dalpha = dL/da~ opacity_r / sqrt(det Sigma_2d), and Eq. 10:
    dI/da~ = exp(.); for one Gaussian, dL/dalpha = sum_p G I / alpha exactly."""
    mu, sc, alpha, sig = (6.0, 6.0, 3.0), (1.2, 1.9, 2.4), 0.37, 1.1
    z = np.array([1.5, 3.5])
    H, W = 12, 12
    rng = np.random.Generator(np.random.PCG64(3))
    G = rng.standard_normal((2, H, W))
    I = oracle.render(*one(mu, sc, Q_RAND, alpha), z, H, W, sig)
    _, _, _, da = oracle.render_backward(*one(mu, sc, Q_RAND, alpha), z, H, W, sig, G)
    assert da[0] == pytest.approx((G * I).sum() / alpha, rel=1e-12)


def test_voxelize_gradient_finite_differences():
    """P9 for Eq. 12: voxelizer gradient vs central differences."""
    rng = np.random.Generator(np.random.PCG64(44))
    n, X, Y, Z = 4, 10, 9, 8
    mu = np.column_stack([rng.uniform(2, 8, n), rng.uniform(2, 7, n), rng.uniform(2, 6, n)])
    sc = rng.uniform(0.8, 2.0, (n, 3))
    q = rng.standard_normal((n, 4))
    al = rng.uniform(0.2, 1.0, n)
    G = rng.standard_normal((Z, Y, X))
    p = {"mu": mu, "scale": sc, "quat": q, "alpha": al}

    def fwd():
        return oracle.voxelize(mu, sc, q, al, X, Y, Z, scale_mod=1.1)

    dmu, ds, dq, da = oracle.voxelize_backward(mu, sc, q, al, X, Y, Z, G, scale_mod=1.1)
    _fd_check(fwd, p, {"mu": dmu, "scale": ds, "quat": dq, "alpha": da}, G)


def test_mse_gradient():
    """The MSE loss L = mean (I - T)^2 has dL/dI = 2 (I - T) / n; checked by
    central differences of L itself."""
    rng = np.random.Generator(np.random.PCG64(2))
    I = rng.standard_normal(37)
    T = rng.standard_normal(37)
    L, g = oracle.mse(I, T)
    assert L == pytest.approx(np.mean((I - T) ** 2), rel=1e-14)
    for k in (0, 5, 36):
        e = np.zeros_like(I)
        e[k] = 1e-6
        num = (oracle.mse(I + e, T)[0] - oracle.mse(I - e, T)[0]) / 2e-6
        assert g[k] == pytest.approx(num, rel=1e-6)


def test_count_evals_brute_force():
    """The oracle's count of evaluations inside the culling region equals a direct
    per-pixel count with the conditional covariance Sigma_pp - Sigma_pc Sigma_cp / v
    built from scipy rotations (an independent route to Eq. 6-8)."""
    g = synth.small(seed=4, n=30, extent=(20, 20, 8))
    z = synth.slice_positions(range(8))
    eps, sig, H, W = 1e-3, 1.5, 20, 20
    k2 = 2 * math.log(1 / eps)
    xx, yy = pixel_grid(H, W)
    count = 0
    for i in range(g.n):
        Sg = cov(g.scale[i].astype(np.float64), g.quat[i])
        v = Sg[2, 2] + sig * sig
        b = Sg[:2, 2]
        S2 = Sg[:2, :2] - np.outer(b, b) / v
        Ki = np.linalg.inv(S2)
        for zs in z:
            delta = g.mu[i, 2] - zs
            if math.exp(-0.5 * delta * delta / v) < eps:
                continue
            m2 = g.mu[i, :2].astype(np.float64) - b * delta / v
            dx, dy = xx - m2[0], yy - m2[1]
            q = Ki[0, 0] * dx * dx + 2 * Ki[0, 1] * dx * dy + Ki[1, 1] * dy * dy
            count += int((q <= k2).sum())
    assert oracle.count_evals(g.mu, g.scale, g.quat, g.alpha, z, H, W, sig, eps=eps) == count


def test_voxel_count_lattice_points():
    """The voxel-evaluation count is a lattice-point count: a tiny isotropic
    Gaussian on a voxel centre covers that voxel only; with radius k s in
    (1, sqrt 2) it also covers the 6 face neighbours; a large ball holds about
    its volume (4/3) pi (k s)^3 of points."""
    k = math.sqrt(2 * math.log(1e6))
    one = lambda s, m: oracle.count_vox_evals([m], [(s, s, s)], [(1, 0, 0, 0)], [1.0], 40, 40, 40)
    assert one(0.1, (10.5, 10.5, 10.5)) == 1
    assert one(1.2 / k, (10.5, 10.5, 10.5)) == 7
    n = one(3.0, (20.5, 20.5, 20.5))
    assert n == pytest.approx(4.0 / 3.0 * math.pi * (3.0 * k) ** 3, rel=0.02)
    # clipped by the grid: a ball centred on a corner voxel keeps about an eighth
    c = one(3.0, (0.5, 0.5, 0.5))
    assert c == pytest.approx(n / 8, rel=0.15)
