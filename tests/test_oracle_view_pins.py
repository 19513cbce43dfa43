"""Pins of the oracle's general slice orientation (Sec. S1 view matrix [R_c | t]
with R_c an arbitrary rotation, not only an axis permutation).

Each compares the oracle with something independent of its route:

* adaptive quadrature of Eq. 5 along the oblique plane normal, evaluated on
  world points x = R_c^T (x_c - t) with the world-frame Gaussian built from
  scipy rotations, equals the Eq. 9/10 response times
  F = sqrt(2 pi) sigma_z sqrt(det Sigma / (n^T Sigma n + sigma_z^2)),
  n = the plane normal (third row of R_c);
* rotating the whole scene by Q (mu -> Q mu, q -> q_Q * q by a Hamilton
  product written here) and the view by R_c -> R_c Q^T leaves every image
  unchanged;
* an in-plane translation of t by whole pixels shifts the image by whole pixels;
* a slice sums to 2 pi alpha opacity_r, opacity_r = exp(-delta^2 / 2 (n^T Sigma n
  + sigma_z^2)), delta the signed distance of the Gaussian from the plane;
* permutation views reproduce the axis-aligned renders exactly;
* central finite differences of every gradient under an oblique view;
* the evaluation count equals a direct per-pixel count with the conditional
  covariance of R_c Sigma R_c^T.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_20611_b300 import synth

TWO_PI = 2.0 * math.pi


def rot_wxyz(q):
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def cov(scale, q_wxyz):
    R = rot_wxyz(q_wxyz)
    S = np.diag(np.asarray(scale, np.float64))
    return R @ S @ S @ R.T


def hamilton(a, b):
    """Quaternion product a * b, both (w, x, y, z)."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def random_rotation(seed):
    return Rotation.random(random_state=seed).as_matrix()


def view_through(R, centre, pixel):
    """t such that the world point `centre` lands at camera (pixel[0], pixel[1], 0)."""
    return np.array([pixel[0], pixel[1], 0.0]) - R @ np.asarray(centre, np.float64)


def one(mu, scale, quat, alpha):
    return (np.array([mu], np.float64), np.array([scale], np.float64),
            np.array([quat], np.float64), np.array([alpha], np.float64))


Q1 = np.array([0.62, -0.31, 0.55, 0.46])
Q1 /= np.linalg.norm(Q1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oblique_quadrature_of_eq5(seed):
    R = random_rotation(seed)
    mu = np.array([6.4, 7.1, 5.3])
    sc = (1.1, 2.6, 1.7)
    alpha, sig = 0.75, 1.3
    Sig = cov(sc, Q1)
    K = np.linalg.inv(Sig)
    nrm = R[2]
    F = math.sqrt(TWO_PI) * sig * math.sqrt(np.linalg.det(Sig) / (nrm @ Sig @ nrm + sig * sig))
    t = view_through(R, mu, (6.0, 5.5))
    z = np.array([-1.5, 0.25, 2.0])
    H, W = 12, 12
    I = oracle.render(*one(mu, sc, Q1, alpha), z, H, W, sig, view=(R, t))
    for k, zs in enumerate(z):
        for (iy, ix) in [(1, 2), (5, 6), (7, 4), (10, 9), (3, 11)]:
            xc, yc = ix + 0.5, iy + 0.5

            def integrand(s):
                xw = R.T @ (np.array([xc, yc, zs + s]) - t)
                d = xw - mu
                return math.exp(-s * s / (2 * sig * sig)) * alpha * math.exp(-0.5 * d @ K @ d)

            val, _ = integrate.quad(integrand, -60, 60, epsabs=1e-15, epsrel=1e-12, limit=200)
            assert I[k, iy, ix] * F == pytest.approx(val, rel=1e-9, abs=1e-16)


def test_scene_rotation_invariance():
    g = synth.small(seed=21, n=12, extent=(20, 20, 12))
    Q = random_rotation(9)
    qQ = Rotation.from_matrix(Q).as_quat()  # (x, y, z, w)
    qQ = np.array([qQ[3], qQ[0], qQ[1], qQ[2]])
    R = random_rotation(4)
    t = view_through(R, (10, 10, 6), (12, 11))
    z = np.array([-2.0, 0.5, 3.0])
    mu = g.mu.astype(np.float64)
    q = g.quat.astype(np.float64)
    a = oracle.render(mu, g.scale, q, g.alpha, z, 24, 22, 1.7, view=(R, t))
    mu2 = mu @ Q.T
    q2 = np.array([hamilton(qQ, qi) for qi in q])
    b = oracle.render(mu2, g.scale, q2, g.alpha, z, 24, 22, 1.7, view=(R @ Q.T, t))
    assert a.max() > 1e-3
    np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-13 * a.max())


def test_in_plane_translation_shifts_by_whole_pixels():
    g = synth.small(seed=22, n=10, extent=(16, 16, 10))
    R = random_rotation(5)
    t = view_through(R, (8, 8, 5), (10, 9))
    z = np.array([0.0, 1.5])
    a = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 24, 26, 2.0, view=(R, t))
    b = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 24, 26, 2.0, view=(R, t + np.array([3.0, 2.0, 0.0])))
    np.testing.assert_allclose(b[:, 2:, 3:], a[:, :-2, :-3], rtol=1e-12, atol=1e-300)


def test_oblique_slice_mass():
    mu, sc, alpha, sig = np.array([24.3, 23.8, 12.0]), (1.5, 3.0, 2.0), 0.6, 2.0
    Sig = cov(sc, Q1)
    R = random_rotation(7)
    nrm = R[2]
    v = nrm @ Sig @ nrm + sig * sig
    t = view_through(R, mu, (24.0, 24.0))
    z = np.array([-3.0, 0.0, 2.5])
    I = oracle.render(*one(mu, sc, Q1, alpha), z, 48, 48, sig, view=(R, t))
    for k, zs in enumerate(z):
        delta = (R @ mu + t)[2] - zs
        assert I[k].sum() == pytest.approx(TWO_PI * alpha * math.exp(-0.5 * delta * delta / v), rel=1e-9)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_permutation_views_match_axes(axis):
    g = synth.small(seed=23, n=25, extent=(18, 18, 14))
    perm = {2: (0, 1, 2), 1: (0, 2, 1), 0: (1, 2, 0)}[axis]
    P = np.zeros((3, 3))
    for j in range(3):
        P[j, perm[j]] = 1.0
    z = np.array([2.5, 7.0, 11.5])
    a = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 18, 18, 1.5, axis=axis)
    b = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 18, 18, 1.5, view=(P, np.zeros(3)))
    assert np.array_equal(a, b)


def test_oblique_gradient_finite_differences():
    rng = np.random.Generator(np.random.PCG64(301))
    n, H, W = 5, 12, 14
    mu = np.column_stack([rng.uniform(3, 11, n), rng.uniform(3, 9, n), rng.uniform(1, 5, n)])
    sc = rng.uniform(0.8, 2.2, (n, 3))
    q = rng.standard_normal((n, 4)) * 1.3
    al = rng.uniform(0.2, 1.0, n)
    R = random_rotation(11)
    t = view_through(R, (7, 6, 3), (7, 6))
    z = np.array([-1.0, 0.5, 1.75])
    sig = 1.4
    G = rng.standard_normal((len(z), H, W))
    view = (R, t)

    def fwd():
        return oracle.render(mu, sc, q, al, z, H, W, sig, scale_mod=1.1, view=view)

    dmu, ds, dq, da = oracle.render_backward(mu, sc, q, al, z, H, W, sig, G, scale_mod=1.1, view=view)
    grads = {"mu": dmu, "scale": ds, "quat": dq, "alpha": da}
    for name, arr in {"mu": mu, "scale": sc, "quat": q, "alpha": al}.items():
        flat = arr.reshape(-1)
        num = np.zeros_like(flat)
        for k in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[k]))
            old = flat[k]
            flat[k] = old + h
            lp = float((G * fwd()).sum())
            flat[k] = old - h
            lm = float((G * fwd()).sum())
            flat[k] = old
            num[k] = (lp - lm) / (2 * h)
        scale = max(np.abs(num).max(), 1e-12)
        np.testing.assert_allclose(grads[name].reshape(-1), num, rtol=2e-6, atol=2e-6 * scale,
                                   err_msg=f"gradient of {name}")


def test_oblique_count_brute_force():
    g = synth.small(seed=24, n=30, extent=(20, 20, 8))
    R = random_rotation(13)
    t = view_through(R, (10, 10, 4), (10, 10))
    z = np.array([-2.0, 0.0, 1.5, 3.0])
    eps, sig, H, W = 1e-3, 1.5, 20, 20
    k2 = 2 * math.log(1 / eps)
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    count = 0
    for i in range(g.n):
        Sc = R @ cov(g.scale[i].astype(np.float64), g.quat[i]) @ R.T
        mc = R @ g.mu[i].astype(np.float64) + t
        v = Sc[2, 2] + sig * sig
        b = Sc[:2, 2]
        Ki = np.linalg.inv(Sc[:2, :2] - np.outer(b, b) / v)
        for zs in z:
            delta = mc[2] - zs
            if math.exp(-0.5 * delta * delta / v) < eps:
                continue
            m2 = mc[:2] - b * delta / v
            dx, dy = xx - m2[0], yy - m2[1]
            count += int((Ki[0, 0] * dx * dx + 2 * Ki[0, 1] * dx * dy + Ki[1, 1] * dy * dy <= k2).sum())
    assert oracle.count_evals(g.mu, g.scale, g.quat, g.alpha, z, H, W, sig, eps=eps, view=(R, t)) == count


def test_views_are_validated():
    g = synth.small(seed=25, n=3, extent=(8, 8, 8))
    z = np.array([1.0])
    for R in (2.0 * np.eye(3), np.array([[1, 0.1, 0], [0, 1, 0], [0, 0, 1.0]]), np.full((3, 3), np.nan)):
        with pytest.raises(ValueError):
            oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 8, 8, 1.0, view=(R, np.zeros(3)))
    with pytest.raises(ValueError):
        oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 8, 8, 1.0, view=(np.eye(3), np.array([0, np.inf, 0])))
