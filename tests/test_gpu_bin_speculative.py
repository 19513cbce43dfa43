"""GPU tests of speculative binning.

A render or backward on a context that already holds pair buffers emits and
sorts its (Gaussian, slice, tile) pairs into those buffers' capacity (at most
a quarter more than the context's last pair count) before the pair count comes
back to the host, and checks the count once its rasteriser is queued; a count
that does not fit bins the call again with the count read first and repeats the
rasteriser.  These tests drive every branch: counts that fit, counts that
overflow (a small scene, then a much larger one on the same context), a call
with no pairs at all, and the backward binning on its own.  Each result must be
bitwise equal to the same call on a fresh context (whose first binning always
reads its count first), with the same pair count, and agree with the FP64
oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, rel_l2

pytestmark = pytest.mark.gpu


def scene(seed, n, ext, S, H, W):
    g = synth.small(seed=seed, n=n, extent=ext)
    z = (np.linspace(0.5, ext[2] - 0.5, S)).astype(np.float32)
    G = synth.random_field(seed + 1, (S, H, W))
    return g, z, G, H, W


def orc(g):
    return g.mu, g.scale, g.quat, g.alpha


def fresh_render(g, z, H, W, sigma):
    c = B.Context(0, deterministic=True)
    out = B.gp_render_slices(c, dev_set(g), z, H, W, sigma).cpu().numpy()
    return out, c.last_counts()[0]


def fresh_backward(g, z, H, W, sigma, G):
    c = B.Context(0, deterministic=True)
    gr = B.gp_render_backward(c, dev_set(g), z, H, W, sigma, torch.from_numpy(G).cuda())
    return [t.cpu().numpy() for t in gr]


def test_counts_that_fit_and_counts_that_overflow():
    c = B.Context(0, deterministic=True)
    small = scene(11, 40, (24, 24, 8), 2, 24, 24)
    big = scene(12, 3000, (96, 80, 40), 12, 80, 96)
    mid = scene(13, 2500, (96, 80, 40), 12, 80, 96)
    for k, (g, z, G, H, W) in enumerate((small, big, mid, big, small, big)):
        out = B.gp_render_slices(c, dev_set(g), z, H, W, 2.0).cpu().numpy()
        pairs = c.last_counts()[0]
        ref, ref_pairs = fresh_render(g, z, H, W, 2.0)
        assert pairs == ref_pairs, f"call {k}: {pairs} pairs, fresh context {ref_pairs}"
        assert np.array_equal(out, ref), f"call {k}: image differs from a fresh context's"
        if k in (1, 2):
            assert_forward_close(out, oracle.render(*orc(g), z, H, W, 2.0), f"call {k}")


def test_backward_binning_overflow():
    c = B.Context(0, deterministic=True)  # reuse_bins off: every backward bins its own call
    small = scene(21, 40, (24, 24, 8), 2, 24, 24)
    big = scene(22, 3000, (96, 80, 40), 12, 80, 96)
    for k, (g, z, G, H, W) in enumerate((small, big, big)):
        gr = B.gp_render_backward(c, dev_set(g), z, H, W, 2.0, torch.from_numpy(G).cuda())
        ref = fresh_backward(g, z, H, W, 2.0, G)
        for name, a, r in zip(("mu", "scale", "quat", "alpha"), gr, ref):
            assert np.array_equal(a.cpu().numpy(), r), f"call {k}: d{name} differs from a fresh context's"
        if k == 1:
            gref = oracle.render_backward(*orc(g), z, H, W, 2.0, G)
            assert_grads_close(gr, gref, "overflowed backward")


def test_no_pairs_after_pairs():
    """A speculative call whose Gaussians reach none of its planes: the image is
    zero everywhere and the gradients are zero."""
    c = B.Context(0, deterministic=True)
    g, z, G, H, W = scene(31, 500, (48, 48, 16), 4, 48, 48)
    B.gp_render_slices(c, dev_set(g), z, H, W, 2.0)
    far = np.array([5000.0, 6000.0], np.float32)
    out = B.gp_render_slices(c, dev_set(g), far, H, W, 2.0).cpu().numpy()
    assert c.last_counts()[0] == 0
    assert not np.any(out)
    gr = B.gp_render_backward(c, dev_set(g), far, H, W, 2.0, torch.ones(2, H, W, device="cuda"))
    for a in gr:
        assert not torch.any(a)


def _half(g, sl):
    return synth.GaussianSet(g.mu[sl], g.scale[sl], g.quat[sl], g.alpha[sl], g.extent)


def test_more_than_a_million_gaussians_split_in_halves():
    """1.2M Gaussians (the per-warp pair totals then take the multi-kernel scan):
    the image agrees with the FP64 oracle on sampled pixels as closely as the
    two halves rendered apart and added, and every Gaussian's gradient is the
    one its half gives (it depends only on dL/dI and that Gaussian) within
    rounding: the units of a Gaussian fall in other lanes of the tile's rounds
    when its neighbours in the list differ, so the order of its per-tile sums
    may change.  Each pixel sums about 25k terms in fp32 (1.2M Gaussians of
    about 195 pixels each over 96 x 96 pixels), so the sampled error bound is
    that of such sums, and the full render must be as close to the oracle as
    the halves are."""
    n = 1_200_000
    g = synth.small(seed=41, n=n, extent=(96, 96, 8))
    z = np.array([2.5, 5.5], np.float32)
    H = W = 96
    G = synth.random_field(42, (2, H, W))
    c = B.Context(0, deterministic=True)
    full = B.gp_render_slices(c, dev_set(g), z, H, W, 1.5).cpu().numpy().astype(np.float64)
    grads = [t.cpu().numpy() for t in B.gp_render_backward(c, dev_set(g), z, H, W, 1.5, torch.from_numpy(G).cuda())]
    parts, pgrads = 0.0, []
    for sl in (slice(0, n // 2), slice(n // 2, n)):
        h = _half(g, sl)
        c2 = B.Context(0, deterministic=True)
        parts = parts + B.gp_render_slices(c2, dev_set(h), z, H, W, 1.5).cpu().numpy().astype(np.float64)
        pgrads.append([t.cpu().numpy() for t in
                       B.gp_render_backward(c2, dev_set(h), z, H, W, 1.5, torch.from_numpy(G).cuda())])
    rng = np.random.default_rng(43)
    s_idx, iy, ix = rng.integers(0, 2, 256), rng.integers(0, H, 256), rng.integers(0, W, 256)
    ref = oracle.render_points(*orc(g), z, 1.5, s_idx, ix + 0.5, iy + 0.5)
    e_full = rel_l2(full[s_idx, iy, ix], ref)
    e_parts = rel_l2(parts[s_idx, iy, ix], ref)
    assert e_full <= 5e-5 and e_full <= 2.0 * e_parts + 1e-6, (e_full, e_parts)
    assert rel_l2(full, parts) <= 1e-4
    for k, name in enumerate(("mu", "scale", "quat", "alpha")):
        joined = np.concatenate([pgrads[0][k], pgrads[1][k]], axis=0)
        assert rel_l2(grads[k], joined) <= 1e-5, f"d{name}"
