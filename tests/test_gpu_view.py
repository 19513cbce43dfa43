"""GPU parity of oblique slice stacks (general view [R_c | t], Sec. S1) against
the FP64 oracle: forward and backward at several orientations with ragged
image sizes, bitwise identity of permutation views with the axis-aligned
calls, bin reuse across views, batched and served oblique requests, autograd,
argument checks, and a full-size microscopy stack on sampled pixels."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, np32, rel_l2

pytestmark = pytest.mark.gpu


def orc(g):
    return g.mu, g.scale, g.quat, g.alpha


def oblique(seed, centre, pixel):
    """A random rotation (fp32-exact) and the t that puts `centre` at camera (pixel, 0)."""
    R = Rotation.random(random_state=seed).as_matrix().astype(np.float32).astype(np.float64)
    t = np.array([pixel[0], pixel[1], 0.0]) - R @ np.asarray(centre, np.float64)
    return R, t.astype(np.float32).astype(np.float64)


def perm_view(axis):
    P = np.zeros((3, 3))
    for j, w in enumerate({2: (0, 1, 2), 1: (0, 2, 1), 0: (1, 2, 0)}[axis]):
        P[j, w] = 1.0
    return P, np.zeros(3)


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


@pytest.mark.parametrize("seed,H,W", [(1, 72, 61), (2, 48, 96), (3, 33, 17)])
def test_oblique_forward_matches_oracle(ctx, seed, H, W):
    g = synth.small(seed=40 + seed, n=1500, extent=(64, 64, 32))
    view = oblique(seed, (32, 32, 16), (W / 2, H / 2))
    z = np.array([-9.0, -2.5, 0.0, 3.25, 11.0], np.float32)
    out = B.gp_render_slices(ctx, dev_set(g), z, H, W, 2.0, view=view)
    ref = oracle.render(*orc(g), z, H, W, 2.0, view=view)
    assert ref.max() > 0.05
    assert_forward_close(np32(out), ref, f"oblique view {seed}")


@pytest.mark.parametrize("seed", [4, 5])
def test_oblique_backward_matches_oracle(seed):
    c = B.Context(0, deterministic=bool(seed % 2))
    g = synth.small(seed=50 + seed, n=400, extent=(40, 40, 20))
    view = oblique(seed, (20, 20, 10), (22, 19))
    H, W = 44, 38
    z = np.array([-4.0, -1.0, 2.5, 6.0], np.float32)
    G = synth.random_field(60 + seed, (len(z), H, W))
    grads = B.gp_render_backward(c, dev_set(g), z, H, W, 1.8, torch.from_numpy(G).cuda(), view=view)
    ref = oracle.render_backward(*orc(g), z, H, W, 1.8, G, view=view)
    assert_grads_close(grads, ref, f"oblique backward {seed}")


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_permutation_view_is_bitwise_the_axis_call(ctx, axis):
    g = synth.small(seed=61, n=800, extent=(48, 48, 48))
    gs = dev_set(g)
    z = synth.slice_positions([3, 17, 30, 44])
    a = B.gp_render_slices(ctx, gs, z, 48, 48, 2.5, axis=axis)
    b = B.gp_render_slices(ctx, gs, z, 48, 48, 2.5, view=perm_view(axis))
    c = B.gp_render_slices(ctx, gs, z, 48, 48, 2.5, view=B.view_from_axis(axis))
    assert torch.equal(a, b) and torch.equal(a, c)
    dctx = B.Context(0, deterministic=True)
    G = torch.from_numpy(synth.random_field(62, (4, 48, 48))).cuda()
    ga = B.gp_render_backward(dctx, gs, z, 48, 48, 2.5, G, axis=axis)
    gb = B.gp_render_backward(dctx, gs, z, 48, 48, 2.5, G, view=perm_view(axis))
    for x, y in zip(ga, gb):
        assert torch.equal(x, y)


def test_bins_are_reused_only_for_the_same_view():
    g = synth.small(seed=63, n=600, extent=(40, 40, 20))
    gs = dev_set(g)
    z = np.array([-2.0, 1.0, 4.0], np.float32)
    v1 = oblique(6, (20, 20, 10), (20, 20))
    v2 = oblique(7, (20, 20, 10), (20, 20))
    G = torch.from_numpy(synth.random_field(64, (3, 40, 40))).cuda()
    reuse = B.Context(0, deterministic=True, reuse_bins=True)
    fresh = B.Context(0, deterministic=True, reuse_bins=False)
    B.gp_render_slices(reuse, gs, z, 40, 40, 2.0, view=v1)
    a = B.gp_render_backward(reuse, gs, z, 40, 40, 2.0, G, view=v1)   # reuses v1's bins
    b = B.gp_render_backward(reuse, gs, z, 40, 40, 2.0, G, view=v2)   # must not reuse them
    a_ref = B.gp_render_backward(fresh, gs, z, 40, 40, 2.0, G, view=v1)
    b_ref = B.gp_render_backward(fresh, gs, z, 40, 40, 2.0, G, view=v2)
    for x, y in zip(a, a_ref):
        assert torch.equal(x, y)
    for x, y in zip(b, b_ref):
        assert torch.equal(x, y)


def test_oblique_eval_count_matches_oracle(ctx):
    g = synth.small(seed=65, n=1200, extent=(64, 64, 32))
    view = oblique(8, (32, 32, 16), (32, 32))
    z = np.linspace(-10, 10, 6).astype(np.float32)
    ev = B.gp_count_evals(ctx, dev_set(g), z, 64, 64, 2.0, view=view)
    ref = oracle.count_evals(*orc(g), z, 64, 64, 2.0, view=view)
    # culling decisions are taken in FP32 on the device and FP64 in the oracle:
    # only pixels within rounding of the ellipse boundary may differ
    assert abs(ev - ref) <= 1e-4 * ref


def test_autograd_with_a_view():
    c = B.Context(0, deterministic=True)
    g = synth.small(seed=66, n=300, extent=(32, 32, 16))
    gs = dev_set(g)
    params = [t.clone().requires_grad_(True) for t in (gs.mu, gs.scale, gs.quat, gs.alpha)]
    view = oblique(9, (16, 16, 8), (16, 16))
    z = np.array([-1.0, 2.0], np.float32)
    I = B.render(c, *params, z, 32, 32, 1.5, view=view)
    G = torch.from_numpy(synth.random_field(67, (2, 32, 32))).cuda()
    (I * G).sum().backward()
    ref = B.gp_render_backward(c, gs, z, 32, 32, 1.5, G, view=view)
    for p, r in zip(params, ref):
        assert torch.equal(p.grad, r)


def test_bad_views_are_rejected(ctx):
    gs = dev_set(synth.small(seed=68, n=10, extent=(8, 8, 8)))
    z = np.array([1.0], np.float32)
    for R, t in ((2.0 * np.eye(3), np.zeros(3)), (np.array([[1, 0.1, 0], [0, 1, 0], [0, 0, 1.0]]), np.zeros(3)),
                 (np.full((3, 3), np.nan), np.zeros(3)), (np.eye(3), np.array([0.0, np.inf, 0.0]))):
        with pytest.raises(B.GPError) as ei:
            B.gp_render_slices(ctx, gs, z, 8, 8, 1.0, view=(R, t))
        assert ei.value.status == B.GP_ERR_ARG
    with pytest.raises(B.GPError):
        B.view_from_axis(3)


def test_batch_items_with_views_match_plain_calls():
    ctx = B.Context(0)
    items, refs = [], []
    for k in range(4):
        g = synth.small(seed=70 + k, n=300 + 150 * k, extent=(40, 40, 20))
        gs = dev_set(g)
        z = np.array([-3.0, 0.5, 4.0], np.float32) if k % 2 == 0 else synth.slice_positions([2, 9, 15])
        it = {"gs": gs, "z": z, "H": 40, "W": 36, "sigma_z": 1.5 + 0.5 * k, "axis": 2,
              "out": torch.empty(3, 40, 36, device="cuda"),
              "dL_dI": torch.from_numpy(synth.random_field(80 + k, (3, 40, 36))).cuda(),
              "grads": (torch.empty(gs.n, 3, device="cuda"), torch.empty(gs.n, 3, device="cuda"),
                        torch.empty(gs.n, 4, device="cuda"), torch.empty(gs.n, device="cuda"))}
        if k % 2 == 0:
            it["view"] = oblique(10 + k, (20, 20, 10), (18, 20))
        items.append(it)
        refs.append(g)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    for it, g in zip(items, refs):
        v = it.get("view")
        img = B.gp_render_slices(ctx, it["gs"], it["z"], 40, 36, it["sigma_z"], view=v)
        assert rel_l2(np32(it["out"]), np32(img)) < 1e-6
        gr = B.gp_render_backward(ctx, it["gs"], it["z"], 40, 36, it["sigma_z"], it["dL_dI"], view=v)
        for a, b in zip(it["grads"], gr):
            assert rel_l2(np32(a), np32(b)) < 1e-4
        if v is not None:
            assert_forward_close(np32(it["out"]), oracle.render(*orc(g), it["z"], 40, 36, it["sigma_z"], view=v),
                                 "batched oblique")
    plan.close()


def test_served_oblique_slices_batch_and_match_plain():
    ctx = B.Context(0)
    g = synth.small(seed=90, n=2000, extent=(96, 96, 48))
    gs = dev_set(g)
    srv = B.Server(ctx, workers=1, max_batch_slices=64)
    sid = srv.load_set(gs)
    view = oblique(12, (48, 48, 24), (48, 48))
    rng = np.random.Generator(np.random.PCG64(91))
    zs = [rng.uniform(-20, 20, 1).astype(np.float32) for _ in range(10)]
    outs = [torch.empty(1, 96, 96, device="cuda") for _ in zs]
    tickets = [srv.submit(B.GP_REQ_SLICE, sid, o, z=z, H=96, W=96, sigma_z=2.0, view=view) for z, o in zip(zs, outs)]
    # an axis-aligned request between them is never batched with the oblique ones
    ax_out = torch.empty(1, 96, 96, device="cuda")
    t_ax = srv.submit(B.GP_REQ_SLICE, sid, ax_out, z=np.array([20.0], np.float32), H=96, W=96, sigma_z=2.0)
    res = []
    for t in tickets + [t_ax]:
        for _ in range(600):
            r = srv.poll(t, timeout_ms=100)
            if r is not None:
                res.append(r)
                break
    assert len(res) == len(tickets) + 1 and all(r["status"] == B.GP_OK for r in res)
    for z, o in zip(zs, outs):
        assert torch.equal(o, B.gp_render_slices(ctx, gs, z, 96, 96, 2.0, view=view))
    assert torch.equal(ax_out, B.gp_render_slices(ctx, gs, np.array([20.0], np.float32), 96, 96, 2.0))
    ref = oracle.render(*orc(g), np.concatenate(zs), 96, 96, 2.0, view=view)
    assert_forward_close(np.concatenate([np32(o) for o in outs]), ref, "served oblique")
    srv.close()


def test_microscopy_oblique_stack_sampled():
    """500k Gaussians in 1024 x 1024 x 256: an oblique 16-plane stack of 1024^2
    through the volume's centre, checked on 1,024 sampled pixels."""
    c = B.Context(0)
    g = synth.microscopy()
    view = oblique(14, (512, 512, 128), (512, 512))
    z = np.linspace(-60, 60, 16).astype(np.float32)
    out = B.gp_render_slices(c, dev_set(g), z, 1024, 1024, 3.0, view=view)
    rng = np.random.Generator(np.random.PCG64(15))
    ps = np.repeat(np.arange(16), 64).astype(np.int32)
    iy = rng.integers(0, 1024, ps.size)
    ix = rng.integers(0, 1024, ps.size)
    ref = oracle.render_points(*orc(g), z, 3.0, ps, ix + 0.5, iy + 0.5, view=view)
    got = np32(out[torch.from_numpy(ps).long(), torch.from_numpy(iy), torch.from_numpy(ix)])
    assert ref.max() > 0.0
    assert_forward_close(got, ref, "microscopy oblique sampled")
