"""FP64 oracle of the photometric loss L = L1 + lambda * D-SSIM (Eq. 11,
lambda = 0.2 in Sec. 5.1) and its gradient with respect to the rendered slices.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product).

Readings (the paper names the terms but prints neither):
* L1 = mean |I - T| over every pixel of every slice; its gradient takes
  sign(0) = 0.
* SSIM is the structural similarity of Wang et al. (2004) computed per slice
  with an 11 x 11 Gaussian window of standard deviation 1.5 (normalised to sum
  1), C1 = (0.01 R)^2, C2 = (0.03 R)^2 with data range R = 1, and zero padding at
  the image borders (the window is not renormalised there -- the convention of
  the Gaussian-splatting code the paper builds on):
      SSIM(p) = (2 mu_I mu_T + C1)(2 s_IT + C2) / ((mu_I^2 + mu_T^2 + C1)(s_I^2 + s_T^2 + C2))
  with mu, s the window-weighted means, variances and covariance at p;
  D-SSIM = 1 - mean over pixels and slices of SSIM(p).
* The loss is the paper's sum as printed, L = L1 + lambda D-SSIM.

The window sums use scipy.ndimage.correlate (zero padding) as a library step;
the gradient is the chain rule written out: with m_I = G*I, m_II = G*I^2,
m_IT = G*(I T) the window moments,
    d mean(SSIM) / dI = (1/n) [ G*(dS/dm_I) + 2 I G*(dS/dm_II) + T G*(dS/dm_IT) ],
the window being symmetric, so that the adjoint of G* is G* (zero padding).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The normalised 11 x 11 Gaussian window (outer product of the 1-D one)."""
    x = np.arange(WIN, dtype=np.float64) - (WIN // 2)
    g = np.exp(-x * x / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def _conv(a, Wn):
    return ndimage.correlate(a, Wn, mode="constant", cval=0.0)


def ssim_map(I, T):
    """SSIM(p) of one slice (2-D arrays)."""
    Wn = window()
    I = np.asarray(I, np.float64)
    T = np.asarray(T, np.float64)
    mI, mT = _conv(I, Wn), _conv(T, Wn)
    sII = _conv(I * I, Wn) - mI * mI
    sTT = _conv(T * T, Wn) - mT * mT
    sIT = _conv(I * T, Wn) - mI * mT
    num = (2 * mI * mT + C1) * (2 * sIT + C2)
    den = (mI * mI + mT * mT + C1) * (sII + sTT + C2)
    return num / den


def l1_dssim(I, T, lam=0.2):
    """(L, L1, mean SSIM, dL/dI) for stacks I, T of shape [S, H, W]."""
    I = np.asarray(I, np.float64)
    T = np.asarray(T, np.float64)
    n = I.size
    Wn = window()
    L1 = float(np.abs(I - T).mean())
    g = np.sign(I - T) / n
    ssum = 0.0
    for s in range(I.shape[0]):
        X, Y = I[s], T[s]
        mI, mT = _conv(X, Wn), _conv(Y, Wn)
        mII, mTT, mIT = _conv(X * X, Wn), _conv(Y * Y, Wn), _conv(X * Y, Wn)
        sII, sTT, sIT = mII - mI * mI, mTT - mT * mT, mIT - mI * mT
        A = 2 * mI * mT + C1
        Bv = 2 * sIT + C2
        Cv = mI * mI + mT * mT + C1
        D = sII + sTT + C2
        S = A * Bv / (Cv * D)
        ssum += float(S.sum())
        # partial derivatives of S with respect to the variables (mI, sII, sIT)
        dS_dmI = (2 * mT * Bv) / (Cv * D) - S * (2 * mI) / Cv
        dS_dsII = -S / D
        dS_dsIT = 2 * A / (Cv * D)
        # ... and with respect to the window moments (m_I, m_II, m_IT)
        d_mI = dS_dmI + dS_dsII * (-2 * mI) + dS_dsIT * (-mT)
        d_mII = dS_dsII
        d_mIT = dS_dsIT
        dssim = _conv(d_mI, Wn) + 2 * X * _conv(d_mII, Wn) + Y * _conv(d_mIT, Wn)
        g[s] += -lam * dssim / n
    mean_ssim = ssum / n
    return L1 + lam * (1.0 - mean_ssim), L1, mean_ssim, g


__all__ = ["WIN", "SIGMA", "C1", "C2", "window", "ssim_map", "l1_dssim"]
