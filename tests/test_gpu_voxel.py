"""GPU parity of the differentiable voxelizer (Eq. 12) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, np32

pytestmark = pytest.mark.gpu


def orc(g):
    return (g.mu, g.scale, g.quat, g.alpha)


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return B.Context(0)


def test_voxelize_ragged_full(ctx):
    """400 Gaussians on a 41 x 35 x 27 grid (no dimension a multiple of 8)."""
    g = synth.small(seed=40, n=400, extent=(41, 35, 27))
    vol = B.gp_voxelize(ctx, dev_set(g, 1.2), 41, 35, 27)
    ref = oracle.voxelize(*orc(g), 41, 35, 27, scale_mod=1.2)
    assert_forward_close(np32(vol), ref, "voxelize")


@pytest.mark.parametrize("det", [False, True])
def test_voxelize_backward(det):
    c = B.Context(0, deterministic=det)
    g = synth.small(seed=41, n=300, extent=(30, 26, 22))
    G = synth.random_field(8, (22, 26, 30))
    grads = B.gp_voxelize_backward(c, dev_set(g), 30, 26, 22, torch.from_numpy(G).cuda())
    ref = oracle.voxelize_backward(*orc(g), 30, 26, 22, G)
    assert_grads_close(grads, ref, f"voxelize backward det={det}")
    if det:
        again = B.gp_voxelize_backward(c, dev_set(g), 30, 26, 22, torch.from_numpy(G).cuda())
        for a, b in zip(grads, again):
            assert torch.equal(a, b)


def test_voxelize_empty_and_outside(ctx):
    e = B.GaussianSet(torch.zeros(0, 3, device="cuda"), torch.ones(0, 3, device="cuda"),
                      torch.zeros(0, 4, device="cuda"), torch.zeros(0, device="cuda"))
    assert B.gp_voxelize(ctx, e, 9, 9, 9).abs().max().item() == 0.0
    g = synth.small(seed=42, n=20, extent=(8, 8, 8))
    g.mu = (g.mu - np.float32(400.0)).astype(np.float32)
    assert B.gp_voxelize(ctx, dev_set(g), 9, 9, 9).abs().max().item() == 0.0


def test_voxelize_serving_size_sampled(ctx):
    """A 256^3 voxelize of 100k Gaussians (the serving request size), on sampled voxels."""
    g = synth.small(seed=43, n=100_000, extent=(256, 256, 256))
    vol = B.gp_voxelize(ctx, dev_set(g), 256, 256, 256)
    rng = np.random.Generator(np.random.PCG64(44))
    idx = rng.integers(0, 256, (512, 3))
    ref = oracle.voxelize_points(*orc(g), idx[:, 0] + 0.5, idx[:, 1] + 0.5, idx[:, 2] + 0.5)
    got = np32(vol[torch.from_numpy(idx[:, 2]), torch.from_numpy(idx[:, 1]), torch.from_numpy(idx[:, 0])])
    assert_forward_close(got, ref, "voxelize 256^3 sampled")


def test_voxel_eval_count_matches_oracle():
    """gp_count_vox_evals (double-precision row intervals) against the oracle's
    brute-force lattice count; only voxels within rounding of an ellipsoid's
    boundary may differ."""
    c = B.Context(0)
    g = synth.small(seed=77, n=300, extent=(40, 36, 28))
    got = B.gp_count_vox_evals(c, dev_set(g), 40, 36, 28)
    ref = oracle.count_vox_evals(g.mu, g.scale, g.quat, g.alpha, 40, 36, 28)
    assert ref > 0 and abs(got - ref) <= 1e-4 * ref
