"""Pins of the culling bounds in ``tests/truncation.py`` (the tolerance the
random sweep uses where the parity bars are tighter than what culling may
drop).

* Its closed form of every term, summed, equals the oracle's brute-force render
  on the three slice axes and an oblique view, with a scale modifier.
* Its forward bound is the whole image where every pair is axially culled, zero
  inside a lone Gaussian's culling ellipse, and carries eps of the image's mass
  for a Gaussian wide against the pixel grid (a Gaussian's mass beyond
  Mahalanobis radius k is exp(-k^2/2) = eps of it).
* Its gradient bound holds for the oracle's own gradient of the culled terms:
  for one Gaussian, the oracle's backward with dL/dI zeroed inside the ellipse
  is the gradient of exactly those terms.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_20611_b300 import synth
from tests import truncation


def small(seed, n, extent):
    return synth.small(seed=seed, n=n, extent=extent)


@pytest.mark.parametrize("axis", [0, 1, 2, "oblique"])
def test_closed_form_equals_oracle(axis):
    g = small(71, 50, (20, 20, 20))
    z = np.array([1.5, 6.0, 10.25, 18.0])
    o = (g.mu, g.scale, g.quat, g.alpha)
    if axis == "oblique":
        R = Rotation.random(random_state=4).as_matrix()
        view = (R, np.array([10.0, 10.0, 0.0]) - R @ np.array([10.0, 10.0, 10.0]))
        ref = oracle.render(*o, z, 21, 19, 2.5, scale_mod=1.3, view=view)
    else:
        view = truncation.axis_view(axis)
        ref = oracle.render(*o, z, 21, 19, 2.5, axis=axis, scale_mod=1.3)
    got = truncation.render_closed_form(g, z, 21, 19, 2.5, 1.3, view)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def _one(mu, scale, quat, alpha):
    class G:
        pass
    g = G()
    g.mu, g.scale = np.array([mu], np.float64), np.array([scale], np.float64)
    g.quat, g.alpha = np.array([quat], np.float64), np.array([alpha], np.float64)
    return g


def test_forward_bound_special_cases():
    q = np.array([0.8, 0.3, -0.2, 0.4])
    # the plane is far from the Gaussian: opacity_r < eps, everything is culled
    far = _one((10.0, 9.0, 40.0), (1.5, 2.0, 1.0), q, 0.7)
    z = np.array([2.0])
    img = oracle.render(far.mu, far.scale, far.quat, far.alpha, z, 20, 20, 1.0)
    b = truncation.forward_bound(far, z, 20, 20, 1.0)
    np.testing.assert_allclose(b, img, rtol=1e-12, atol=0)
    # a wide Gaussian on the plane: nothing near its centre is culled, and the
    # culled mass is eps of the image's
    wide = _one((32.0, 31.0, 5.0), (3.5, 5.0, 2.0), q, 0.7)
    z = np.array([5.5])
    img = oracle.render(wide.mu, wide.scale, wide.quat, wide.alpha, z, 64, 64, 1.0)
    b = truncation.forward_bound(wide, z, 64, 64, 1.0)
    assert b[0, 26:38, 26:38].max() == 0.0
    assert b.sum() == pytest.approx(1e-6 * img.sum(), rel=0.1)
    b9 = truncation.forward_bound(wide, z, 64, 64, 1.0, eps=1e-9)
    assert b9.sum() == pytest.approx(1e-9 * img.sum(), rel=0.15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_bound_holds_for_the_oracles_culled_gradient(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    g = _one(rng.uniform(8, 16, 3), rng.uniform(0.6, 2.5, 3), q, rng.uniform(0.2, 1.0))
    z = np.array([4.0, 11.5, 12.0, 19.0])
    H, W = 24, 22
    G = rng.standard_normal((z.size, H, W))
    mask = truncation.forward_bound(g, z, H, W, 1.7) > 0  # one Gaussian: its culled pixels
    o = (g.mu, g.scale, g.quat, g.alpha)
    culled = oracle.render_backward(*o, z, H, W, 1.7, G * mask)
    bounds = truncation.gradient_bound(g, z, H, W, 1.7, G)
    for c, bb in zip(culled, bounds):
        c = np.asarray(c).reshape(bb.shape)
        assert np.all(np.abs(c) <= bb * (1 + 1e-9) + 1e-300), (c, bb)
    # and it is not vacuous: with dL/dI of one sign per pixel matching the
    # culled alpha term, the bound on alpha is attained
    culled_pos = oracle.render_backward(*o, z, H, W, 1.7, np.abs(G) * mask)
    assert abs(float(np.asarray(culled_pos[3]).reshape(-1)[0])) == pytest.approx(
        float(bounds[3][0]) / 1.01, rel=1e-9)
