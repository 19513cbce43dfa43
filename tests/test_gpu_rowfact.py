"""GPU parity of the row-factored rasterisers (GP_EXP_POLY_ROW: two exp2 per
row of 8 pixels, powers of the per-pixel step by multiplication, the quadratic
part once per Gaussian and tile) with the FP64 oracle, forward and backward, on
the small workload, ragged images through every axis and both tile sizes, a set
whose scales span 0.05 to 30 pixels (narrow Gaussians take the per-pixel
fallback, wide and elongated ones give rows with large and small steps), the
deterministic mode, a batched plan and the full-size microscopy workload on
sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, np32, rel_l2

pytestmark = pytest.mark.gpu


def orc(g):
    return (g.mu, g.scale, g.quat, g.alpha)


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0, exp_mode=B.GP_EXP_POLY_ROW)


def wide_range_set(seed, n, extent, lo=0.05, hi=30.0):
    """Scales log-uniform in [lo, hi] pixels per axis, so the set holds
    needles, discs and blobs in every orientation."""
    g = synth.small(seed=seed, n=n, extent=extent)
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    g.scale = np.exp(rng.uniform(np.log(lo), np.log(hi), (n, 3))).astype(np.float32)
    return g


def test_forward_small_full(ctx):
    g = synth.small()
    z = synth.slice_positions(range(32))
    out = B.gp_render_slices(ctx, dev_set(g), z, 64, 64, 2.0)
    ref = oracle.render(*orc(g), z, 64, 64, 2.0)
    assert_forward_close(np32(out), ref, "row-factored small")
    # a few ulp per pixel: well inside the bar
    assert rel_l2(np32(out), ref) < 2e-6


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("tile", [16, 8])
def test_forward_ragged_axes_tiles(axis, tile):
    c = B.Context(0, tile=tile, exp_mode=B.GP_EXP_POLY_ROW)
    g = synth.small(seed=77, n=400, extent=(45, 40, 37))
    z = np.array([20.3, 3.5, 33.0, 11.75, 0.5], np.float32)
    out = B.gp_render_slices(c, dev_set(g), z, 37, 45, 1.7, axis)
    ref = oracle.render(*orc(g), z, 37, 45, 1.7, axis=axis)
    assert_forward_close(np32(out), ref, f"row axis {axis} tile {tile}")


def test_forward_scales_from_discs_to_blobs(ctx):
    """Scales 0.3 to 30 pixels: every Gaussian takes the factored rows, with
    steps from near 0 (wide) to far beyond the fp32 range (elongated ones far
    from a row's vertex)."""
    g = wide_range_set(101, 700, (48, 40, 20), lo=0.3)
    z = synth.slice_positions(range(0, 20, 3))
    out = B.gp_render_slices(ctx, dev_set(g), z, 40, 48, 1.2)
    ref = oracle.render(*orc(g), z, 40, 48, 1.2)
    assert_forward_close(np32(out), ref, "row wide-range scales")


def test_forward_needles_match_the_per_pixel_form(ctx):
    """Scales down to 0.05 pixel: needles are ill-conditioned in fp32 (a
    rounding of 1e-6 pixel in the projected centre moves exp(-d^2 / 2 s^2) by
    d / s^2 * 1e-6, 1e-4 relative here), so neither form meets the 1e-5 bar on
    them; the row form, whose narrow Gaussians take the per-pixel exp2, must
    not add error to what the per-pixel form already has."""
    g = wide_range_set(103, 700, (48, 40, 20))
    z = synth.slice_positions(range(0, 20, 3))
    ref = oracle.render(*orc(g), z, 40, 48, 1.2)
    row = rel_l2(np32(B.gp_render_slices(ctx, dev_set(g), z, 40, 48, 1.2)), ref)
    poly = rel_l2(np32(B.gp_render_slices(B.Context(0), dev_set(g), z, 40, 48, 1.2)), ref)
    assert row <= 1.1 * poly + 1e-6, (row, poly)


def test_backward_small_full(ctx):
    g = synth.small()
    tgt = synth.small(seed=2001)
    z = synth.slice_positions(range(32))
    T = oracle.render(*orc(tgt), z, 64, 64, 2.0)
    gs = dev_set(g)
    I = B.gp_render_slices(ctx, gs, z, 64, 64, 2.0)
    dL, _ = B.gp_mse_grad(ctx, I, torch.from_numpy(T.astype(np.float32)).cuda())
    grads = B.gp_render_backward(ctx, gs, z, 64, 64, 2.0, dL)
    I_ref = oracle.render(*orc(g), z, 64, 64, 2.0)
    _, G_ref = oracle.mse(I_ref, T.astype(np.float32))
    ref = oracle.render_backward(*orc(g), z, 64, 64, 2.0, G_ref)
    assert_grads_close(grads, ref, "row-factored small")


@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("tile,det", [(16, False), (16, True), (8, False)])
def test_backward_ragged(axis, tile, det):
    c = B.Context(0, tile=tile, deterministic=det, exp_mode=B.GP_EXP_POLY_ROW)
    g = synth.small(seed=88, n=300, extent=(29, 35, 26))
    z = np.array([7.25, 1.5, 20.0, 13.5], np.float32)
    G = synth.random_field(5, (len(z), 26, 29))
    grads = B.gp_render_backward(c, dev_set(g, 1.1), z, 26, 29, 1.4, torch.from_numpy(G).cuda(), axis)
    ref = oracle.render_backward(*orc(g), z, 26, 29, 1.4, G, axis=axis, scale_mod=1.1)
    assert_grads_close(grads, ref, f"row axis {axis} tile {tile} det {det}")


def test_backward_scales_from_discs_to_blobs(ctx):
    g = wide_range_set(102, 500, (40, 36, 16), lo=0.3)
    z = synth.slice_positions(range(0, 16, 2))
    G = synth.random_field(9, (len(z), 36, 40))
    grads = B.gp_render_backward(ctx, dev_set(g), z, 36, 40, 1.3, torch.from_numpy(G).cuda())
    ref = oracle.render_backward(*orc(g), z, 36, 40, 1.3, G)
    assert_grads_close(grads, ref, "row wide-range scales")


def test_backward_needles_match_the_per_pixel_form(ctx):
    g = wide_range_set(104, 500, (40, 36, 16))
    z = synth.slice_positions(range(0, 16, 2))
    G = synth.random_field(10, (len(z), 36, 40))
    ref = oracle.render_backward(*orc(g), z, 36, 40, 1.3, G)
    Gd = torch.from_numpy(G).cuda()
    row = B.gp_render_backward(ctx, dev_set(g), z, 36, 40, 1.3, Gd)
    poly = B.gp_render_backward(B.Context(0), dev_set(g), z, 36, 40, 1.3, Gd)
    for name, a, b, r in zip(("mu", "scale", "quat", "alpha"), row, poly, ref):
        ea, eb = rel_l2(np32(a), r), rel_l2(np32(b), r)
        assert ea <= max(1.1 * eb + 1e-6, 1e-3), (name, ea, eb)


def test_deterministic_mode_is_bitwise_repeatable():
    c = B.Context(0, deterministic=True, exp_mode=B.GP_EXP_POLY_ROW)
    g = synth.small(seed=21, n=1500, extent=(64, 48, 24))
    z = synth.slice_positions(range(24))
    G = torch.from_numpy(synth.random_field(6, (24, 48, 64))).cuda()
    gs = dev_set(g)
    r1 = [t.clone() for t in B.gp_render_backward(c, gs, z, 48, 64, 2.0, G)]
    r2 = [t.clone() for t in B.gp_render_backward(c, gs, z, 48, 64, 2.0, G)]
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    o1 = B.gp_render_slices(c, gs, z, 48, 64, 2.0).clone()
    o2 = B.gp_render_slices(c, gs, z, 48, 64, 2.0)
    assert torch.equal(o1, o2)


def test_batched_plan_matches_oracle():
    c = B.Context(0, exp_mode=B.GP_EXP_POLY_ROW)
    sets = [synth.small(seed=300 + k, n=200 + 150 * k, extent=(40, 32, 12)) for k in range(3)]
    zs = [synth.slice_positions(range(k, 12, 3)) for k in range(3)]
    items = []
    for g, z in zip(sets, zs):
        items.append(dict(gs=dev_set(g), z=z, H=32, W=40, sigma_z=1.5,
                          out=torch.empty(len(z), 32, 40, device="cuda")))
    plan = B.BatchPlan(c, items, autotune=False)
    plan.run()
    torch.cuda.synchronize()
    for g, z, it in zip(sets, zs, items):
        ref = oracle.render(*orc(g), z, 32, 40, 1.5)
        assert_forward_close(np32(it["out"]), ref, "row batched")


def test_per_thread_kernels_reject_the_row_mode():
    with pytest.raises(B.GPError):
        B.Context(0, exp_mode=B.GP_EXP_POLY_ROW, fwd_px=2)


def test_microscopy_full_size_sampled():
    """500k Gaussians, 1024^2, 16 of 256 slices, sigma_z = 3, as the bench
    renders them with the row mode: 1,024 sampled pixels and 24 sampled
    Gaussians' gradients against the oracle."""
    c = B.Context(0, exp_mode=B.GP_EXP_POLY_ROW, reuse_bins=True)
    g = synth.microscopy()
    idx = synth.slice_batch(7, 256, 256, 16)
    z = synth.slice_positions(idx)
    gs = dev_set(g)
    out = B.gp_render_slices(c, gs, z, 1024, 1024, 3.0)
    rng = np.random.Generator(np.random.PCG64(11))
    ps = np.repeat(np.arange(16), 64).astype(np.int32)
    iy, ix = rng.integers(0, 1024, ps.size), rng.integers(0, 1024, ps.size)
    ref = oracle.render_points(*orc(g), z, 3.0, ps, ix + 0.5, iy + 0.5)
    got = np32(out[torch.from_numpy(ps).long(), torch.from_numpy(iy), torch.from_numpy(ix)])
    assert_forward_close(got, ref, "row microscopy sampled")
    G = synth.random_field(12, (16, 1024, 1024))
    grads = B.gp_render_backward(c, gs, z, 1024, 1024, 3.0, torch.from_numpy(G).cuda())
    near = np.where(np.min(np.abs(g.mu[:, 2][:, None] - z[None, :]), axis=1) < 6.0)[0]
    pick = np.sort(np.random.Generator(np.random.PCG64(13)).choice(near, 24, replace=False))
    ref = oracle.render_backward(g.mu[pick], g.scale[pick], g.quat[pick], g.alpha[pick], z, 1024, 1024, 3.0, G)
    sub = [t[torch.from_numpy(pick).long().cuda()] for t in grads]
    assert_grads_close(sub, ref, "row microscopy sampled grads")
