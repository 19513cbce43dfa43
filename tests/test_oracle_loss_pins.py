"""Pins of the L1 + lambda D-SSIM oracle (Eq. 11) against things other than its
own route: a brute-force per-pixel window sum for SSIM (no convolution
routine), the identity SSIM(I, I) = 1 with zero gradient, the closed form of
two constant images away from the borders, the window's own properties, and
central finite differences of the loss."""
import math

import numpy as np
import pytest

from oracle import loss


def test_window_is_a_normalised_separable_gaussian():
    Wn = loss.window()
    assert Wn.shape == (11, 11) and Wn.sum() == pytest.approx(1.0, abs=1e-15)
    assert Wn[5, 5] / Wn[5, 6] == pytest.approx(math.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-12)
    assert np.allclose(Wn, Wn.T) and np.allclose(Wn, Wn[::-1, ::-1])


def test_ssim_map_equals_brute_force_window_sums():
    rng = np.random.Generator(np.random.PCG64(1))
    I = rng.uniform(0, 1, (13, 17))
    T = np.clip(I + 0.2 * rng.standard_normal(I.shape), 0, 1)
    S = loss.ssim_map(I, T)
    x = np.arange(11) - 5
    g = np.exp(-x * x / (2 * 1.5 ** 2))
    g /= g.sum()
    for (py, px) in [(0, 0), (6, 8), (12, 16), (3, 14), (9, 1)]:
        mI = mT = mII = mTT = mIT = 0.0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                y, xx = py + dy, px + dx
                if 0 <= y < 13 and 0 <= xx < 17:
                    w = g[dy + 5] * g[dx + 5]
                    a, b = I[y, xx], T[y, xx]
                    mI += w * a; mT += w * b; mII += w * a * a; mTT += w * b * b; mIT += w * a * b
        sI, sT, sIT = mII - mI * mI, mTT - mT * mT, mIT - mI * mT
        ref = ((2 * mI * mT + 1e-4) * (2 * sIT + 9e-4)) / ((mI ** 2 + mT ** 2 + 1e-4) * (sI + sT + 9e-4))
        assert S[py, px] == pytest.approx(ref, rel=1e-12)


def test_identical_images():
    rng = np.random.Generator(np.random.PCG64(2))
    I = rng.uniform(0, 1, (2, 20, 24))
    L, L1, ms, g = loss.l1_dssim(I, I.copy())
    assert L1 == 0.0 and ms == pytest.approx(1.0, abs=1e-14) and L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(g).max() < 1e-15  # SSIM is at its maximum; sign(0) = 0


def test_constant_images_closed_form():
    a, b = 0.3, 0.7
    I = np.full((1, 32, 32), a)
    T = np.full((1, 32, 32), b)
    S = loss.ssim_map(I[0], T[0])
    ref = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)  # variances vanish away from the borders
    np.testing.assert_allclose(S[5:-5, 5:-5], ref, rtol=1e-12)


def test_gradient_by_finite_differences():
    rng = np.random.Generator(np.random.PCG64(3))
    I = rng.uniform(0.05, 0.95, (2, 9, 11))
    T = np.clip(I + 0.3 * rng.standard_normal(I.shape), 0, 1)
    _, _, _, g = loss.l1_dssim(I, T, lam=0.2)
    for idx in [(0, 0, 0), (0, 4, 5), (1, 8, 10), (1, 2, 7), (0, 6, 1)]:
        e = np.zeros_like(I)
        e[idx] = 1e-7
        num = (loss.l1_dssim(I + e, T)[0] - loss.l1_dssim(I - e, T)[0]) / 2e-7
        assert g[idx] == pytest.approx(num, rel=1e-5, abs=1e-12)
