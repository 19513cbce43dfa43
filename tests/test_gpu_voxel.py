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


# ------------------------------------------------ the plane-stack voxelizer

def test_voxelize_matches_the_voxelizer_limit_of_the_slice_operator(ctx):
    """Pin P4 on the device: each z-plane of the volume is the slice of that
    plane at sigma_z -> 0 times sqrt(det Sigma_cond) (the slice operator's
    amplitude alpha / sqrt(det Sigma_2d) against the voxelizer's alpha), here
    checked through the oracle's slice render at a tiny sigma_z for a single
    Gaussian."""
    g = synth.small(seed=45, n=1, extent=(24, 20, 12))
    vol = np32(B.gp_voxelize(ctx, dev_set(g), 24, 20, 12))
    z = synth.slice_positions(range(12))
    sl = oracle.render(*orc(g), z, 20, 24, 1e-4)
    # sqrt(det Sigma_2d) of the conditional covariance at sigma_z -> 0
    w, x, y, zq = g.quat[0].astype(np.float64) / np.linalg.norm(g.quat[0].astype(np.float64))
    R = np.array([[1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)],
                  [2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)],
                  [2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)]])
    S = R @ np.diag(g.scale[0].astype(np.float64) ** 2) @ R.T
    cond = S[:2, :2] - np.outer(S[:2, 2], S[:2, 2]) / S[2, 2]
    assert_forward_close(vol, sl * np.sqrt(np.linalg.det(cond)), "voxelize = slice limit")


def test_voxelize_single_plane_and_thin_grids(ctx):
    g = synth.small(seed=46, n=150, extent=(19, 23, 1))
    for X, Y, Z in ((19, 23, 1), (1, 23, 5), (19, 1, 3)):
        vol = B.gp_voxelize(ctx, dev_set(g), X, Y, Z)
        assert_forward_close(np32(vol), oracle.voxelize(*orc(g), X, Y, Z), f"grid {X}x{Y}x{Z}")


def test_voxelize_row_factored():
    c = B.Context(0, exp_mode=B.GP_EXP_POLY_ROW)
    g = synth.small(seed=47, n=400, extent=(37, 29, 21))
    vol = B.gp_voxelize(c, dev_set(g), 37, 29, 21)
    assert_forward_close(np32(vol), oracle.voxelize(*orc(g), 37, 29, 21), "voxelize row-factored")
    G = synth.random_field(9, (21, 29, 37))
    grads = B.gp_voxelize_backward(c, dev_set(g), 37, 29, 21, torch.from_numpy(G).cuda())
    assert_grads_close(grads, oracle.voxelize_backward(*orc(g), 37, 29, 21, G), "voxelize backward row-factored")


def test_voxelizer_and_slice_bins_are_never_shared():
    """With bin reuse on, a voxelize after a slice render of the same planes,
    and a slice backward after a voxelize, must each bin again (different
    amplitude and culling): both match the oracle; and the voxelize backward
    right after its forward reuses the bins bitwise (deterministic mode)."""
    c = B.Context(0, reuse_bins=True, deterministic=True)
    plain = B.Context(0, deterministic=True)
    g = synth.small(seed=48, n=300, extent=(26, 22, 14))
    gs = dev_set(g)
    z = synth.slice_positions(range(14))
    G = torch.from_numpy(synth.random_field(10, (14, 22, 26))).cuda()
    B.gp_render_slices(c, gs, z, 22, 26, 1.5)
    gv = B.gp_voxelize_backward(c, gs, 26, 22, 14, G)
    assert_grads_close(gv, oracle.voxelize_backward(*orc(g), 26, 22, 14, G.cpu().numpy()), "vox after slices")
    B.gp_voxelize(c, gs, 26, 22, 14)
    gsl = B.gp_render_backward(c, gs, z, 22, 26, 1.5, G)
    assert_grads_close(gsl, oracle.render_backward(*orc(g), z, 22, 26, 1.5, G.cpu().numpy()), "slices after vox")
    B.gp_voxelize(c, gs, 26, 22, 14)
    reused = [t.clone() for t in B.gp_voxelize_backward(c, gs, 26, 22, 14, G)]
    fresh = B.gp_voxelize_backward(plain, gs, 26, 22, 14, G)
    for a, b in zip(reused, fresh):
        assert torch.equal(a, b)


def test_voxelize_bad_arguments(ctx):
    import ctypes
    g = dev_set(synth.small(seed=49, n=10, extent=(8, 8, 8)))
    s = g.c()
    vol = torch.empty(8, 8, 8, device="cuda")
    for X, Y, Z in ((0, 8, 8), (8, 8, -1), (8, -3, 8)):
        st = B.lib.gp_voxelize(ctx.h, ctypes.byref(s), X, Y, Z, ctypes.c_void_p(vol.data_ptr()), None)
        assert st == B.GP_ERR_ARG, (X, Y, Z, st)
    torch.cuda.synchronize()


def test_voxelize_ultrasound_full_size_sampled():
    """The voxelize benchmark's workload in its launch configuration: 200k
    Gaussians of the ultrasound set on the 512^3 grid, forward on 512 sampled
    voxels, backward against a random dL/dV on 8 sampled Gaussians."""
    c = B.Context(0, reuse_bins=True)
    g = synth.ultrasound()
    gs = dev_set(g)
    vol = B.gp_voxelize(c, gs, 512, 512, 512)
    rng = np.random.Generator(np.random.PCG64(52))
    idx = rng.integers(0, 512, (512, 3))
    ref = oracle.voxelize_points(*orc(g), idx[:, 0] + 0.5, idx[:, 1] + 0.5, idx[:, 2] + 0.5)
    got = np32(vol[torch.from_numpy(idx[:, 2]), torch.from_numpy(idx[:, 1]), torch.from_numpy(idx[:, 0])])
    assert_forward_close(got, ref, "voxelize 512^3 sampled")
    del vol
    G = torch.randn(512, 512, 512, device="cuda", generator=torch.Generator(device="cuda").manual_seed(53))
    grads = B.gp_voxelize_backward(c, gs, 512, 512, 512, G)
    sel = np.sort(rng.choice(g.n, 8, replace=False))
    og = oracle.voxelize_backward(g.mu[sel], g.scale[sel], g.quat[sel], g.alpha[sel], 512, 512, 512, G.cpu().numpy())
    sub = [t[torch.from_numpy(sel).long().cuda()] for t in grads]
    assert_grads_close(sub, og, "voxelize 512^3 sampled grads")
