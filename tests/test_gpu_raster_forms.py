"""GPU tests of the two default rasteriser forms on slice planes (the default,
GP_RASTER_AUTO, takes row units for the forward and for the voxelizer's
backward, block-culled cells for the slice backward; the voxelizer is covered
by test_gpu_voxel.py): block-culled (GP_RASTER_BLOCK) and row units
(GP_RASTER_ROWS, one warp per tile; on 16 x 16 tiles each lane of the forward
owns one 8-pixel row segment), forward and
backward against the FP64 oracle on every slice axis, an oblique view, both
tile sizes and both exponentials; the row units' deterministic backward is
bitwise repeatable, and the two forms agree with each other within rounding.
The evaluated-pixel count of the row units covers every pixel inside the
culling ellipses (it is at least the algorithmic count) and is below the
block-culled cells' pixel count."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, rel_l2

pytestmark = pytest.mark.gpu

FORMS = [B.GP_RASTER_BLOCK, B.GP_RASTER_ROWS]


def orc(g):
    return g.mu, g.scale, g.quat, g.alpha


def _oblique():
    rng = np.random.Generator(np.random.PCG64(31))
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    t = np.array([20.0, 18.0, 0.0]) - q @ np.array([20.0, 17.0, 13.0])
    return q.astype(np.float32), t.astype(np.float32)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("view", [0, 1, 2, "oblique"])
@pytest.mark.parametrize("tile", [16, 8])
def test_forms_against_oracle(form, view, tile):
    """Five planes of 37 x 43: with 16 x 16 tiles that is 45 (plane, tile)
    keys, an odd count, so the row backward's last CTA (two tiles per CTA)
    has a warp without a tile."""
    c = B.Context(0, tile=tile, raster=form)
    g = synth.small(seed=404, n=400, extent=(41, 35, 27))
    gs = dev_set(g, 1.15)
    z = np.array([3.25, 11.0, 0.5, 19.75, 26.0], np.float32)
    H, W = 37, 43
    G = synth.random_field(77, (len(z), H, W))
    kw = dict(view=_oblique()) if view == "oblique" else dict(axis=view)
    okw = dict(view=_oblique()) if view == "oblique" else dict(axis=view)
    out = B.gp_render_slices(c, gs, z, H, W, 1.7, **kw)
    ref = oracle.render(*orc(g), z, H, W, 1.7, scale_mod=1.15, **okw)
    assert_forward_close(out.cpu().numpy(), ref, f"form {form} view {view} tile {tile}")
    grads = B.gp_render_backward(c, gs, z, H, W, 1.7, torch.from_numpy(G).cuda(), **kw)
    gref = oracle.render_backward(*orc(g), z, H, W, 1.7, G, scale_mod=1.15, **okw)
    assert_grads_close(grads, gref, f"form {form} view {view} tile {tile}")


@pytest.mark.parametrize("exp_mode", [B.GP_EXP_POLY, B.GP_EXP_HW])
def test_forms_agree_on_the_small_workload(exp_mode):
    g = synth.small(seed=1001, n=2000, extent=(64, 64, 32))
    gs = dev_set(g)
    z = synth.slice_positions(range(32))
    G = torch.from_numpy(synth.random_field(8, (32, 64, 64))).cuda()
    res = []
    for form in FORMS:
        c = B.Context(0, raster=form, exp_mode=exp_mode)
        res.append((B.gp_render_slices(c, gs, z, 64, 64, 2.0), B.gp_render_backward(c, gs, z, 64, 64, 2.0, G)))
    (ia, ga), (ib, gb) = res
    assert rel_l2(ia.cpu().numpy(), ib.cpu().numpy()) < 1e-6
    for a, b in zip(ga, gb):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-5


def test_row_units_deterministic_backward_is_bitwise_repeatable():
    c = B.Context(0, raster=B.GP_RASTER_ROWS, deterministic=True)
    g = synth.small(seed=21, n=1500, extent=(64, 48, 24))
    gs = dev_set(g)
    z = synth.slice_positions(range(24))
    G = torch.from_numpy(synth.random_field(6, (24, 48, 64))).cuda()
    a = B.gp_render_backward(c, gs, z, 48, 64, 2.0, G)
    b = B.gp_render_backward(c, gs, z, 48, 64, 2.0, G)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    i1 = B.gp_render_slices(c, gs, z, 48, 64, 2.0)
    i2 = B.gp_render_slices(B.Context(0, raster=B.GP_RASTER_ROWS), gs, z, 48, 64, 2.0)
    assert torch.equal(i1, i2)  # the forward's order does not depend on the backward mode


def test_evaluated_count_bounds():
    c = B.Context(0, raster=B.GP_RASTER_ROWS)
    g = synth.small(seed=1001, n=2000, extent=(64, 64, 32))
    gs = dev_set(g)
    z = synth.slice_positions(range(32))
    B.gp_render_slices(c, gs, z, 64, 64, 2.0)
    pairs = c.last_counts()[0]
    alg = B.gp_count_evals(c, gs, z, 64, 64, 2.0)
    ev, evb = B.gp_count_evaluated(c, gs, z, 64, 64, 2.0)
    assert alg <= ev == evb <= pairs * 256
    assert ev % 8 == 0
    blk_f, blk_b = B.gp_count_evaluated(B.Context(0, raster=B.GP_RASTER_BLOCK), gs, z, 64, 64, 2.0)
    assert alg <= blk_b <= blk_f <= pairs * 256 and ev <= blk_b
    vox_alg = B.gp_count_vox_evals(c, gs, 64, 64, 32)
    vox_ev, vox_evb = B.gp_count_vox_evaluated(c, gs, 64, 64, 32)
    assert vox_alg <= vox_ev == vox_evb and vox_ev % 8 == 0
