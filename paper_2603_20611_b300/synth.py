"""Seeded synthetic inputs for the slice projection operator.

This module only draws random numbers: it holds none of the operator's
arithmetic, so both the CUDA path and the FP64 oracle can consume its output
(the same bytes) without sharing any code.  Every draw comes from numpy's PCG64
generator with an explicit seed.

The workloads stand in for the paper's datasets (TDSC-ABUS, rDL-LSM,
Tribolium, hiPSC, TNNI1; Sec. 5 "Dataset"), none of which is used here:

* ``small``       -- 2,000 Gaussians in a 64 x 64 x 32 volume, sigma_z = 2,
                     all 32 slices;
* ``microscopy``  -- 500k Gaussians in a 1024 x 1024 x 256 light-sheet-like
                     stack, z-scale 3x the xy-scale, sparse log-normal
                     intensities, sigma_z = 3, random batches of 16 slices;
* ``ultrasound``  -- 200k Gaussians in 512^3, sigma_z = 5, all 512 slices,
                     Rayleigh speckle times smooth blobs as the target;
* ``batched``     -- 64 uneven sets;
* ``serving``     -- 8 resident sets of 50k-2M Gaussians.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class GaussianSet:
    """Structure-of-arrays Gaussian parameters (Sec. S1: G = (mu, s, q, alpha))."""
    mu: np.ndarray      # [n, 3] float32, world units (voxels)
    scale: np.ndarray   # [n, 3] float32, linear, > 0
    quat: np.ndarray    # [n, 4] float32, (w, x, y, z), unit norm
    alpha: np.ndarray   # [n]    float32
    extent: tuple = (0, 0, 0)  # (X, Y, Z) of the volume the set lives in

    @property
    def n(self) -> int:
        return int(self.alpha.shape[0])

    def subset(self, idx) -> "GaussianSet":
        return GaussianSet(self.mu[idx].copy(), self.scale[idx].copy(), self.quat[idx].copy(),
                           self.alpha[idx].copy(), self.extent)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions: a normalised 4-D standard normal."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def small_law_set(rng, n, extent, log_scale_mean=math.log(1.5), log_scale_std=0.3):
    """Means uniform over the volume, log-scales ~ N(log 1.5, 0.3) per axis,
    uniform rotations, intensities ~ U(0, 1)."""
    X, Y, Z = extent
    mu = rng.uniform(0.0, 1.0, (n, 3)) * np.array([X, Y, Z], np.float64)
    scale = np.exp(rng.normal(log_scale_mean, log_scale_std, (n, 3)))
    quat = uniform_quaternions(rng, n)
    alpha = rng.uniform(0.0, 1.0, n)
    return GaussianSet(mu.astype(np.float32), scale.astype(np.float32), quat,
                       alpha.astype(np.float32), tuple(extent))


def small(seed: int = 1001, n: int = 2000, extent=(64, 64, 32)) -> GaussianSet:
    return small_law_set(_rng(seed), n, extent)


def microscopy(seed: int = 1002, n: int = 500_000, extent=(1024, 1024, 256)) -> GaussianSet:
    """Light-sheet-shaped set: s_x, s_y ~ exp(N(log 2, 0.4)) drawn independently,
    s_z = 3 sqrt(s_x s_y); intensities clip(LogNormal(-2, 1), 0, 1)."""
    rng = _rng(seed)
    X, Y, Z = extent
    mu = rng.uniform(0.0, 1.0, (n, 3)) * np.array([X, Y, Z], np.float64)
    sxy = np.exp(rng.normal(math.log(2.0), 0.4, (n, 2)))
    sz = 3.0 * np.sqrt(sxy[:, 0] * sxy[:, 1])
    scale = np.concatenate([sxy, sz[:, None]], axis=1)
    quat = uniform_quaternions(rng, n)
    alpha = np.clip(rng.lognormal(-2.0, 1.0, n), 0.0, 1.0)
    return GaussianSet(mu.astype(np.float32), scale.astype(np.float32), quat,
                       alpha.astype(np.float32), tuple(extent))


def ultrasound(seed: int = 1003, n: int = 200_000, extent=(512, 512, 512)) -> GaussianSet:
    return small_law_set(_rng(seed), n, extent)


def slice_batch(seed: int, n_slices: int, depth: int, k: int) -> np.ndarray:
    """k distinct slice indices out of n_slices, ascending (one random batch)."""
    rng = _rng(seed)
    return np.sort(rng.choice(n_slices, size=k, replace=False)).astype(np.int32)


def slice_positions(indices) -> np.ndarray:
    """Plane position of slice index s: the centre of voxel layer s, s + 0.5."""
    return (np.asarray(indices, np.float64) + 0.5).astype(np.float32)


def speckle_blob_target(seed: int, shape, n_blobs: int = 16) -> np.ndarray:
    """Ultrasound-like target [Z, Y, X]: Rayleigh(1) speckle times a sum of smooth
    isotropic blobs (std U(20, 80) voxels, centres uniform), scaled to [0, 1]."""
    rng = _rng(seed)
    Z, Y, X = shape
    z = np.arange(Z, dtype=np.float32) + 0.5
    y = np.arange(Y, dtype=np.float32) + 0.5
    x = np.arange(X, dtype=np.float32) + 0.5
    env = np.zeros(shape, np.float32)
    for _ in range(n_blobs):
        c = rng.uniform(0.0, 1.0, 3) * np.array([X, Y, Z])
        sd = rng.uniform(20.0, 80.0)
        gz = np.exp(-0.5 * ((z - c[2]) / sd) ** 2).astype(np.float32)
        gy = np.exp(-0.5 * ((y - c[1]) / sd) ** 2).astype(np.float32)
        gx = np.exp(-0.5 * ((x - c[0]) / sd) ** 2).astype(np.float32)
        env += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    speck = rng.rayleigh(1.0, shape).astype(np.float32)
    t = speck * env
    t /= t.max()
    return t


@dataclass
class BatchItem:
    gs: GaussianSet
    H: int
    W: int
    z: np.ndarray          # [S] float32 plane positions
    sigma_z: float


def batched(seed: int = 1004, n_sets: int = 64, depth: int = 64,
            n_range=(1_000, 200_000), sides=(128, 256, 512, 1024),
            slices_range=(8, 64), sigma_range=(1.0, 6.0)) -> list:
    """Uneven sets: counts log-uniform in n_range, square slices of a side drawn
    from ``sides``, 8-64 slices each, sigma_z ~ U(1, 6), small-set laws."""
    rng = _rng(seed)
    items = []
    for k in range(n_sets):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        side = int(rng.choice(np.asarray(sides)))
        S = int(rng.integers(slices_range[0], slices_range[1] + 1))
        sigma = float(rng.uniform(*sigma_range))
        gs = small_law_set(rng, n, (side, side, depth))
        idx = np.sort(rng.choice(depth, size=min(S, depth), replace=False))
        items.append(BatchItem(gs, side, side, slice_positions(idx), sigma))
    return items


def serving_sets(seed: int = 1005, n_sets: int = 8, n_range=(50_000, 2_000_000),
                 extent=(1024, 1024, 1024)) -> list:
    rng = _rng(seed)
    sets = []
    for _ in range(n_sets):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        sets.append(small_law_set(rng, n, extent))
    return sets


def random_field(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Standard-normal field (used as an upstream gradient dL/dI in tests)."""
    return (_rng(seed).standard_normal(shape) * scale).astype(np.float32)
