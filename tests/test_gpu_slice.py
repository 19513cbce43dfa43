"""GPU parity of the slice renderer (K-pre, K-pair, sort, K-range, K-fwd, K-loss,
K-bwd, K-det, K-bwd-pre) against the FP64 oracle, through the C ABI.

Small workloads are compared in full; the full-size microscopy (500k Gaussians,
1024^2, 16 slices) and ultrasound (200k Gaussians, 512^3, 512 slices) workloads
are rendered exactly as bench.py launches them and compared on sampled pixels,
and their gradients on sampled Gaussians (the gradient of one Gaussian depends
only on dL/dI and that Gaussian, so the oracle can compute it alone).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import (assert_forward_close, assert_grads_close, dev_set, np32, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return B.Context(0)


def orc(g):
    return (g.mu, g.scale, g.quat, g.alpha)


# ------------------------------------------------------------------ exp2

# the backward's degree-4 form: its Remez bound 3.6e-6 plus a few fp32 roundings
@pytest.mark.parametrize("mode,tol", [(B.GP_EXP_POLY, 2.5e-7), (B.GP_EXP_HW, 2e-6), (B.GP_EXP_POLY_GRAD, 4e-6)])
def test_exp2_accuracy(ctx, mode, tol):
    """The rasterisers' exp2 against FP64 over its whole domain [-125, 0.5]."""
    rng = np.random.Generator(np.random.PCG64(1))
    x = np.concatenate([np.linspace(-125.0, 0.5, 1 << 20), rng.uniform(-30, 0.5, 1 << 20)]).astype(np.float32)
    y = B.gp_exp2_eval(ctx, torch.from_numpy(x).cuda(), mode).cpu().numpy().astype(np.float64)
    ref = np.exp2(x.astype(np.float64))
    rel = np.abs(y / ref - 1.0)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("scalar,packed", [(B.GP_EXP_POLY, B.GP_EXP_POLY_PACKED),
                                           (B.GP_EXP_POLY_GRAD, B.GP_EXP_POLY_GRAD_PACKED)])
def test_packed_exp2_is_bitwise_the_scalar_form(ctx, scalar, packed):
    """The rasterisers evaluate two pixels per packed fp32x2 instruction; every
    lane must round exactly as the scalar exp2 does (odd length: the last
    element pairs with a dummy)."""
    rng = np.random.Generator(np.random.PCG64(2))
    x = torch.from_numpy(np.concatenate([np.linspace(-125.0, 0.5, (1 << 20) + 1),
                                         rng.uniform(-130, 0.5, 4097)]).astype(np.float32)).cuda()
    a = B.gp_exp2_eval(ctx, x, scalar)
    b = B.gp_exp2_eval(ctx, x, packed)
    assert torch.equal(a, b)


def test_exp2_matches_cuda_exp2f(ctx):
    """Cross-check with CUDA's own exp2 (through torch) on the same inputs."""
    x = torch.linspace(-60.0, 0.0, 1 << 18, device="cuda")
    y = B.gp_exp2_eval(ctx, x, B.GP_EXP_POLY)
    ref = torch.exp2(x.double())
    assert (y.double() / ref - 1).abs().max().item() <= 2.5e-7


# ----------------------------------------------------------- forward, small

def test_forward_small_full(ctx):
    """2,000 Gaussians in 64x64x32, sigma_z = 2, all 32 slices: every pixel."""
    g = synth.small()
    z = synth.slice_positions(range(32))
    out = B.gp_render_slices(ctx, dev_set(g), z, 64, 64, 2.0)
    ref = oracle.render(*orc(g), z, 64, 64, 2.0)
    assert_forward_close(np32(out), ref, "small")
    pairs, issued = ctx.last_counts()
    assert pairs > 0 and issued == pairs * 256


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("tile,fpx", [(16, 0), (16, 1), (16, 2), (16, 4), (8, 0), (8, 1), (8, 2)])
def test_forward_ragged_axes_tiles(axis, tile, fpx):
    """Ragged image (37 x 45, not a tile multiple), unsorted and off-centre planes,
    slices through each axis, every tile size and pixels-per-thread variant."""
    c = B.Context(0, tile=tile, fwd_px=fpx)
    g = synth.small(seed=77, n=400, extent=(45, 40, 37))
    z = np.array([20.3, 3.5, 33.0, 11.75, 0.5], np.float32)
    H, W = 37, 45
    out = B.gp_render_slices(c, dev_set(g), z, H, W, 1.7, axis)
    ref = oracle.render(*orc(g), z, H, W, 1.7, axis=axis)
    assert_forward_close(np32(out), ref, f"axis {axis} tile {tile} px {fpx}")


@pytest.mark.parametrize("exp_mode", [B.GP_EXP_HW])
def test_forward_hw_exp(exp_mode):
    """The SFU exponential variant meets the same bar."""
    c = B.Context(0, exp_mode=exp_mode)
    g = synth.small(seed=3, n=600, extent=(48, 48, 16))
    z = synth.slice_positions(range(16))
    out = B.gp_render_slices(c, dev_set(g), z, 48, 48, 2.0)
    assert_forward_close(np32(out), oracle.render(*orc(g), z, 48, 48, 2.0), "hw exp")


def test_forward_scale_mod_and_unnormalised_quats(ctx):
    g = synth.small(seed=5, n=300, extent=(32, 32, 12))
    g.quat = (g.quat * np.linspace(0.3, 3.0, g.n)[:, None]).astype(np.float32)
    z = synth.slice_positions(range(12))
    out = B.gp_render_slices(ctx, dev_set(g, scale_mod=1.3), z, 32, 32, 1.5)
    ref = oracle.render(*orc(g), z, 32, 32, 1.5, scale_mod=1.3)
    assert_forward_close(np32(out), ref, "scale_mod")


def test_forward_edge_cases(ctx):
    g = synth.small(seed=9, n=50, extent=(16, 16, 8))
    z = synth.slice_positions([2, 5])
    # empty set -> zeros
    e = B.GaussianSet(torch.zeros(0, 3, device="cuda"), torch.ones(0, 3, device="cuda"),
                      torch.zeros(0, 4, device="cuda"), torch.zeros(0, device="cuda"))
    out = B.gp_render_slices(ctx, e, z, 16, 16, 1.0)
    assert out.abs().max().item() == 0.0
    # empty stack
    assert B.gp_render_slices(ctx, dev_set(g), np.zeros(0, np.float32), 16, 16, 1.0).shape == (0, 16, 16)
    # every Gaussian far outside the image -> zeros
    far = synth.small(seed=9, n=50, extent=(16, 16, 8))
    far.mu = (far.mu + np.float32(500.0)).astype(np.float32)
    out = B.gp_render_slices(ctx, dev_set(far), z, 16, 16, 1.0)
    assert out.abs().max().item() == 0.0
    # one slice, one pixel row
    out = B.gp_render_slices(ctx, dev_set(g), z[:1], 1, 16, 1.0)
    assert_forward_close(np32(out), oracle.render(*orc(g), z[:1], 1, 16, 1.0), "1 row")
    # degenerate zero-scale Gaussian is culled, the rest still render
    g2 = synth.small(seed=9, n=50, extent=(16, 16, 8))
    g2.scale[0] = 0.0
    out = B.gp_render_slices(ctx, dev_set(g2), z, 16, 16, 1.0)
    keep = np.arange(1, 50)
    ref = oracle.render(g2.mu[keep], g2.scale[keep], g2.quat[keep], g2.alpha[keep], z, 16, 16, 1.0)
    assert_forward_close(np32(out), ref, "zero scale")


def test_bad_arguments_are_rejected(ctx):
    """Argument errors come back as GP_ERR_ARG before any launch."""
    g = dev_set(synth.small(seed=1, n=10, extent=(8, 8, 8)))
    s = g.c()
    out = torch.empty(1, 8, 8, device="cuda")
    z = np.array([1.5], np.float32)
    zn = np.array([np.nan], np.float32)

    def call(S=1, H=8, W=8, sig=1.0, axis=2, zz=z):
        return B.lib.gp_render_slices(ctx.h, ctypes.byref(s), zz.ctypes.data_as(ctypes.c_void_p), S, H, W,
                                      sig, axis, ctypes.c_void_p(out.data_ptr()), None)

    assert call() == B.GP_OK
    for bad in (dict(sig=0.0), dict(sig=float("inf")), dict(axis=3), dict(H=0), dict(S=-1), dict(zz=zn)):
        assert call(**bad) == B.GP_ERR_ARG, bad
    torch.cuda.synchronize()


# ------------------------------------------------------------ loss, small

def test_mse_grad(ctx):
    rng = np.random.Generator(np.random.PCG64(4))
    I = rng.standard_normal((3, 20, 30)).astype(np.float32)
    T = rng.standard_normal((5, 20, 30)).astype(np.float32)
    tidx = [4, 0, 2]
    loss = torch.zeros(1, device="cuda")
    g, _ = B.gp_mse_grad(ctx, torch.from_numpy(I).cuda(), torch.from_numpy(T).cuda(), tidx, loss=loss)
    L, gref = oracle.mse(I, T[tidx])
    np.testing.assert_allclose(np32(g), gref, rtol=1e-6, atol=1e-12)
    assert loss.item() == pytest.approx(L, rel=1e-5)


# ---------------------------------------------------------- backward, small

def small_problem(seed=1001, n=2000, extent=(64, 64, 32), S=32, sigma=2.0):
    g = synth.small(seed=seed, n=n, extent=extent)
    tgt = synth.small(seed=seed + 1000, n=n, extent=extent)
    z = synth.slice_positions(range(S))
    H, W = extent[1], extent[0]
    T = oracle.render(*orc(tgt), z, H, W, sigma)
    return g, z, H, W, sigma, T


def test_backward_small_full(ctx):
    """Full small workload: render, MSE against a target rendered (by the oracle)
    from a second seeded set, backward; compared with the oracle's gradient."""
    g, z, H, W, sig, T = small_problem()
    gs = dev_set(g)
    I = B.gp_render_slices(ctx, gs, z, H, W, sig)
    dL, _ = B.gp_mse_grad(ctx, I, torch.from_numpy(T.astype(np.float32)).cuda())
    grads = B.gp_render_backward(ctx, gs, z, H, W, sig, dL)
    I_ref = oracle.render(*orc(g), z, H, W, sig)
    _, G_ref = oracle.mse(I_ref, T.astype(np.float32))
    ref = oracle.render_backward(*orc(g), z, H, W, sig, G_ref)
    assert_grads_close(grads, ref, "small")


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("tile,bpx", [(16, 0), (16, 2), (16, 4), (16, 8), (8, 0), (8, 2)])
def test_backward_ragged_axes_tiles(axis, tile, bpx):
    c = B.Context(0, tile=tile, bwd_px=bpx)
    g = synth.small(seed=88, n=300, extent=(29, 35, 26))
    z = np.array([7.25, 1.5, 20.0, 13.5], np.float32)
    H, W = 26, 29
    G = synth.random_field(5, (len(z), H, W))
    grads = B.gp_render_backward(c, dev_set(g, 1.1), z, H, W, 1.4, torch.from_numpy(G).cuda(), axis)
    ref = oracle.render_backward(*orc(g), z, H, W, 1.4, G, axis=axis, scale_mod=1.1)
    assert_grads_close(grads, ref, f"axis {axis} tile {tile} px {bpx}")


def test_backward_exponential_keeps_gradients_far_inside_the_bar(ctx):
    """The backward recomputes its exponentials with a degree-4 exp2 (3.6e-6
    relative); on the small workload and a ragged stack its gradients stay
    within 2e-5 relative L2 of the FP64 oracle (measured 1e-6 to 6e-6, as with
    the SFU exponential), fifty times inside the 1e-3 bar."""
    g, z, H, W, sig, T = small_problem()
    gs = dev_set(g)
    I = B.gp_render_slices(ctx, gs, z, H, W, sig)
    dL, _ = B.gp_mse_grad(ctx, I, torch.from_numpy(T.astype(np.float32)).cuda())
    grads = B.gp_render_backward(ctx, gs, z, H, W, sig, dL)
    I_ref = oracle.render(*orc(g), z, H, W, sig)
    _, G_ref = oracle.mse(I_ref, T.astype(np.float32))
    ref = oracle.render_backward(*orc(g), z, H, W, sig, G_ref)
    assert_grads_close(grads, ref, "small", tol=2e-5)
    g2 = synth.small(seed=88, n=300, extent=(29, 35, 26))
    z2 = np.array([7.25, 1.5, 20.0, 13.5], np.float32)
    G2 = synth.random_field(5, (len(z2), 26, 29))
    grads = B.gp_render_backward(ctx, dev_set(g2, 1.1), z2, 26, 29, 1.4, torch.from_numpy(G2).cuda(), 0)
    ref = oracle.render_backward(*orc(g2), z2, 26, 29, 1.4, G2, axis=0, scale_mod=1.1)
    assert_grads_close(grads, ref, "ragged", tol=2e-5)


def test_backward_deterministic_mode_is_bitwise_repeatable():
    cd = B.Context(0, deterministic=True)
    ca = B.Context(0, deterministic=False)
    g = synth.small(seed=21, n=1500, extent=(64, 48, 24))
    z = synth.slice_positions(range(24))
    G = torch.from_numpy(synth.random_field(6, (24, 48, 64))).cuda()
    gs = dev_set(g)
    r1 = [t.clone() for t in B.gp_render_backward(cd, gs, z, 48, 64, 2.0, G)]
    r2 = [t.clone() for t in B.gp_render_backward(cd, gs, z, 48, 64, 2.0, G)]
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    ra = B.gp_render_backward(ca, gs, z, 48, 64, 2.0, G)
    for a, b in zip(r1, ra):
        assert rel_l2(np32(a), np32(b)) < 1e-4
    ref = oracle.render_backward(*orc(g), z, 48, 64, 2.0, G.cpu().numpy())
    assert_grads_close(r1, ref, "deterministic")


def test_autograd_function_matches_backward():
    """The autograd Function routes to gp_render_backward: with the ordered
    (deterministic) reduction both give identical bits."""
    ctx = B.Context(0, deterministic=True)
    g = synth.small(seed=31, n=200, extent=(24, 24, 10))
    z = synth.slice_positions(range(10))
    gs = dev_set(g)
    params = [t.clone().requires_grad_(True) for t in (gs.mu, gs.scale, gs.quat, gs.alpha)]
    I = B.render(ctx, *params, z, 24, 24, 1.5)
    G = torch.from_numpy(synth.random_field(7, (10, 24, 24))).cuda()
    (I * G).sum().backward()
    direct = B.gp_render_backward(ctx, gs, z, 24, 24, 1.5, G)
    for p, d in zip(params, direct):
        assert torch.equal(p.grad, d)


def test_eval_counts(ctx):
    g = synth.small()
    z = synth.slice_positions(range(32))
    ev = B.gp_count_evals(ctx, dev_set(g), z, 64, 64, 2.0)
    pairs, issued = ctx.last_counts()
    assert 0 < ev <= issued


# ------------------------------------------------- full-size, sampled outputs

def _sample_points(seed, S, H, W, per_slice):
    rng = np.random.Generator(np.random.PCG64(seed))
    ps = np.repeat(np.arange(S), per_slice).astype(np.int32)
    iy = rng.integers(0, H, ps.size)
    ix = rng.integers(0, W, ps.size)
    return ps, iy, ix


def test_microscopy_full_size_sampled():
    """500k Gaussians, 1024^2, a random batch of 16 of 256 slices, sigma_z = 3:
    forward on 1,024 sampled pixels, backward on 24 sampled Gaussians."""
    c = B.Context(0)
    g = synth.microscopy()
    idx = synth.slice_batch(7, 256, 256, 16)
    z = synth.slice_positions(idx)
    gs = dev_set(g)
    out = B.gp_render_slices(c, gs, z, 1024, 1024, 3.0)
    ps, iy, ix = _sample_points(11, 16, 1024, 1024, 64)
    ref = oracle.render_points(*orc(g), z, 3.0, ps, ix + 0.5, iy + 0.5)
    got = np32(out[torch.from_numpy(ps).long(), torch.from_numpy(iy), torch.from_numpy(ix)])
    assert_forward_close(got, ref, "microscopy sampled")
    G = synth.random_field(12, (16, 1024, 1024))
    grads = B.gp_render_backward(c, gs, z, 1024, 1024, 3.0, torch.from_numpy(G).cuda())
    rng = np.random.Generator(np.random.PCG64(13))
    # Gaussians that reach the sampled slices (others have zero gradient)
    near = np.where(np.min(np.abs(g.mu[:, 2][:, None] - z[None, :]), axis=1) < 6.0)[0]
    pick = np.sort(rng.choice(near, 24, replace=False))
    ref = oracle.render_backward(g.mu[pick], g.scale[pick], g.quat[pick], g.alpha[pick], z, 1024, 1024,
                                 3.0, G)
    sub = [t[torch.from_numpy(pick).long().cuda()] for t in grads]
    assert_grads_close(sub, ref, "microscopy sampled grads")


def test_ultrasound_full_size_sampled_and_crop():
    """200k Gaussians in 512^3, sigma_z = 5, all 512 slices: forward on sampled
    pixels of 8 slices; backward of a 4,096-Gaussian crop on a 64 x 64 x 32
    window against the oracle's (finite-difference pinned) gradient."""
    c = B.Context(0)
    g = synth.ultrasound()
    z = synth.slice_positions(range(512))
    out = B.gp_render_slices(c, dev_set(g), z, 512, 512, 5.0)
    sl = np.array([0, 77, 150, 255, 256, 311, 430, 511])
    ps, iy, ix = _sample_points(21, len(sl), 512, 512, 48)
    ref = oracle.render_points(*orc(g), z[sl], 5.0, ps, ix + 0.5, iy + 0.5)
    got = np32(out[torch.from_numpy(sl[ps]).long(), torch.from_numpy(iy), torch.from_numpy(ix)])
    assert_forward_close(got, ref, "ultrasound sampled")
    # crop: the 4,096 Gaussians nearest the centre of the window [224,288)^2 x [240,272)
    centre = np.array([256.0, 256.0, 256.0])
    d2 = ((g.mu.astype(np.float64) - centre) ** 2).sum(1)
    crop = g.subset(np.sort(np.argsort(d2)[:4096]))
    crop.mu = (crop.mu - np.array([224, 224, 240], np.float32)).astype(np.float32)
    zc = synth.slice_positions(range(32))
    Tc = synth.random_field(22, (32, 64, 64))
    grads = B.gp_render_backward(c, dev_set(crop), zc, 64, 64, 5.0, torch.from_numpy(Tc).cuda())
    ref = oracle.render_backward(*orc(crop), zc, 64, 64, 5.0, Tc)
    assert_grads_close(grads, ref, "ultrasound crop")


def test_backward_reuses_forward_bins_only_for_identical_calls():
    """reuse_bins: the backward right after a forward with the same arguments
    uses its binning (bitwise the same result in deterministic mode); any other
    call re-bins."""
    g = synth.small(seed=51, n=800, extent=(48, 40, 16))
    z = synth.slice_positions(range(0, 16, 2))
    G = torch.from_numpy(synth.random_field(52, (8, 40, 48))).cuda()
    plain = B.Context(0, deterministic=True)
    reuse = B.Context(0, deterministic=True, reuse_bins=True)
    gs = dev_set(g)
    ref = B.gp_render_backward(plain, gs, z, 40, 48, 2.0, G)
    B.gp_render_slices(reuse, gs, z, 40, 48, 2.0)
    got = B.gp_render_backward(reuse, gs, z, 40, 48, 2.0, G)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    # different planes after the forward: must not reuse
    z2 = (z + np.float32(0.5)).astype(np.float32)
    ref2 = B.gp_render_backward(plain, gs, z2, 40, 48, 2.0, G)
    B.gp_render_slices(reuse, gs, z, 40, 48, 2.0)
    got2 = B.gp_render_backward(reuse, gs, z2, 40, 48, 2.0, G)
    for a, b in zip(got2, ref2):
        assert torch.equal(a, b)


def test_phase_timing_selects_phases():
    """gp_timing_enable_phases times only the chosen phases; gp_timing_enable
    times all of them; bits past the last phase are rejected."""
    c = B.Context(0)
    g = synth.small(seed=77, n=300, extent=(32, 32, 8))
    gs = dev_set(g)
    z = np.array([2.5, 5.5], np.float32)
    G = torch.ones(2, 32, 32, device="cuda")

    def run():
        B.gp_render_slices(c, gs, z, 32, 32, 2.0)
        B.gp_render_backward(c, gs, z, 32, 32, 2.0, G)
        torch.cuda.synchronize()
        return c.timing_read()

    c.timing(True, phases=("fwd",))
    ph = run()
    assert ph["fwd"][2] == 1 and ph["fwd"][0] > 0.0
    assert ph["bin"][2] == 0 and ph["bwd"][2] == 0 and ph["bwd_pre"][2] == 0
    c.timing(True)
    ph = run()
    assert all(ph[p][2] >= 1 for p in ("bin", "fwd", "bwd", "bwd_pre"))
    c.timing(False)
    ph = run()
    assert all(v[2] == 0 for v in ph.values())
    assert B.lib.gp_timing_enable_phases(c.h, 1 << B.GP_NUM_PHASES) == B.GP_ERR_ARG
