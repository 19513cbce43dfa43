"""GPU tests of the batched form: one graph launch renders and differentiates
many uneven Gaussian sets; every item must agree with its own plain launch and
with the FP64 oracle, repeated runs must see updated parameters, and a run that
outgrows the plan must report GP_ERR_OVERFLOW."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, assert_grads_close, dev_set, np32, rel_l2

pytestmark = pytest.mark.gpu


def _items(seed=7, n=6, with_target=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    items, meta = [], []
    for k in range(n):
        side = int(rng.choice([24, 40, 64, 72]))
        depth = int(rng.integers(8, 20))
        cnt = int(rng.integers(50, 600))
        g = synth.small(seed=seed * 100 + k, n=cnt, extent=(side, side + 3, depth))
        S = int(rng.integers(2, 7))
        sig = float(rng.uniform(1.0, 4.0))
        axis = int(rng.integers(0, 3))
        # extent (x, y, z) = (side, side + 3, depth); planes across the slice axis
        span = {2: depth, 1: side + 3, 0: side}[axis]
        z = np.sort(rng.uniform(0.0, span, S)).astype(np.float32)[rng.permutation(S)]
        H, W = {2: (side + 3, side), 1: (depth, side), 0: (depth, side + 3)}[axis]
        gs = dev_set(g)
        it = {"gs": gs, "z": z, "H": H, "W": W, "sigma_z": sig, "axis": axis,
              "out": torch.empty(S, H, W, device="cuda"),
              "grads": (torch.empty(cnt, 3, device="cuda"), torch.empty(cnt, 3, device="cuda"),
                        torch.empty(cnt, 4, device="cuda"), torch.empty(cnt, device="cuda"))}
        if with_target:
            it["target"] = torch.from_numpy(synth.random_field(500 + k, (S, H, W), 0.05)).cuda()
            it["loss"] = torch.zeros(1, device="cuda")
        else:
            it["dL_dI"] = torch.from_numpy(synth.random_field(500 + k, (S, H, W))).cuda()
        items.append(it)
        meta.append(g)
    return items, meta


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_plain_and_oracle(autotune):
    ctx = B.Context(0)
    items, meta = _items()
    plan = B.BatchPlan(ctx, items, autotune=autotune)
    plan.run()
    plan.wait()
    info = plan.info()
    assert info["tile"] in (8, 16) and info["pair_capacity"] > 0
    assert info["fwd_raster"] in ("block", "rows", "pixels") and info["bwd_raster"] in ("block", "rows", "pixels")
    plain = B.Context(0, tile=info["tile"])
    for k, (it, g) in enumerate(zip(items, meta)):
        ref_img = B.gp_render_slices(plain, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["axis"])
        assert rel_l2(np32(it["out"]), np32(ref_img)) < 1e-6, k
        ref_g = B.gp_render_backward(plain, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["dL_dI"],
                                     it["axis"])
        for a, b in zip(it["grads"], ref_g):
            assert rel_l2(np32(a), np32(b)) < 1e-4, k
        if k < 3:
            o = oracle.render(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"],
                              axis=it["axis"])
            assert_forward_close(np32(it["out"]), o, f"batch item {k}")
            og = oracle.render_backward(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"],
                                        it["dL_dI"].cpu().numpy(), axis=it["axis"])
            assert_grads_close(it["grads"], og, f"batch item {k}")
    plan.close()


def test_batch_with_targets_runs_loss_and_backward():
    ctx = B.Context(0)
    items, meta = _items(seed=9, n=4, with_target=True)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    for k, (it, g) in enumerate(zip(items, meta)):
        I = B.gp_render_slices(ctx, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["axis"])
        loss = torch.zeros(1, device="cuda")
        dL, _ = B.gp_mse_grad(ctx, I, it["target"], loss=loss)
        ref = B.gp_render_backward(ctx, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], dL, it["axis"])
        assert it["loss"].item() == pytest.approx(loss.item(), rel=1e-5)
        for a, b in zip(it["grads"], ref):
            assert rel_l2(np32(a), np32(b)) < 1e-4, k
    plan.close()


def test_batch_replay_sees_parameter_updates_and_is_deterministic():
    ctx = B.Context(0, deterministic=True)
    items, meta = _items(seed=11, n=5)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    first = [it["out"].clone() for it in items]
    grads1 = [[t.clone() for t in it["grads"]] for it in items]
    plan.run()
    plan.wait()
    for it, f, g1 in zip(items, first, grads1):
        assert torch.equal(it["out"], f)
        for a, b in zip(it["grads"], g1):
            assert torch.equal(a, b)
    # intensities are linear: doubling alpha in place doubles every image
    for it in items:
        it["gs"].alpha.mul_(2.0)
    plan.run()
    plan.wait()
    for it, f in zip(items, first):
        assert rel_l2(np32(it["out"]), 2.0 * np32(f)) < 1e-6
    plan.close()


def test_batch_overflow_is_reported_not_faulted():
    ctx = B.Context(0)
    items, meta = _items(seed=13, n=6)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    # grow every Gaussian 8x: far more (slice, tile) pairs than the plan holds
    for it in items:
        it["gs"].scale.mul_(8.0)
    plan.run()
    with pytest.raises(B.GPError) as ei:
        plan.wait()
    assert ei.value.status == B.GP_ERR_OVERFLOW
    plan.close()
    # a fresh plan sized for the new parameters runs clean
    plan2 = B.BatchPlan(ctx, items)
    plan2.run()
    plan2.wait()
    plan2.close()


def test_batched_workload_full_size_sampled():
    """The batched benchmark workload itself (64 uneven sets, 1k-200k Gaussians,
    128^2-1024^2 slices, 8-64 planes, sigma_z in [1, 6]) in its benchmarked
    launch configuration (one autotuned plan): for six items, the smallest, the
    largest and four others, forward on 256 sampled pixels and the gradients of
    8 sampled Gaussians against the oracle."""
    ctx = B.Context(0)
    raw = synth.batched()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4004)
    items = []
    for bi in raw:
        S = len(bi.z)
        gs = dev_set(bi.gs)
        items.append({"gs": gs, "z": bi.z, "H": bi.H, "W": bi.W, "sigma_z": bi.sigma_z, "axis": 2,
                      "out": torch.empty(S, bi.H, bi.W, device="cuda"),
                      "dL_dI": torch.randn(S, bi.H, bi.W, device="cuda", generator=gen),
                      "grads": (torch.empty(gs.n, 3, device="cuda"), torch.empty(gs.n, 3, device="cuda"),
                                torch.empty(gs.n, 4, device="cuda"), torch.empty(gs.n, device="cuda"))})
    plan = B.BatchPlan(ctx, items, autotune=True)
    plan.run()
    plan.wait()
    sizes = [bi.gs.n for bi in raw]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 5, 17, 33, 50})
    rng = np.random.Generator(np.random.PCG64(77))
    for k in pick:
        bi, it = raw[k], items[k]
        g, S = bi.gs, len(bi.z)
        ps = rng.integers(0, S, 256).astype(np.int32)
        iy, ix = rng.integers(0, bi.H, 256), rng.integers(0, bi.W, 256)
        ref = oracle.render_points(g.mu, g.scale, g.quat, g.alpha, bi.z, bi.sigma_z, ps, ix + 0.5, iy + 0.5)
        got = np32(it["out"][torch.from_numpy(ps).long(), torch.from_numpy(iy), torch.from_numpy(ix)])
        assert_forward_close(got, ref, f"batched item {k} ({g.n} Gaussians, {S} x {bi.H}^2)")
        near = np.where(np.min(np.abs(g.mu[:, 2][:, None] - bi.z[None, :]), axis=1) < 3.0 * bi.sigma_z + 3.0)[0]
        sel = np.sort(rng.choice(near, min(8, near.size), replace=False))
        og = oracle.render_backward(g.mu[sel], g.scale[sel], g.quat[sel], g.alpha[sel], bi.z, bi.H, bi.W,
                                    bi.sigma_z, it["dL_dI"].cpu().numpy())
        sub = [t[torch.from_numpy(sel).long().cuda()] for t in it["grads"]]
        assert_grads_close(sub, og, f"batched item {k} grads")
    plan.close()


def test_batch_row_units_match_plain_row_units_and_oracle():
    """A plan of a row-unit context (no autotuning) runs the persistent row-unit
    rasterisers; its images and gradients equal the plain row-unit calls'
    bitwise (same per-tile lists and summation order) and the oracle's."""
    ctx = B.Context(0, raster=B.GP_RASTER_ROWS)
    items, meta = _items(seed=11, n=5)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    info = plan.info()
    assert info["fwd_raster"] == "rows" and info["bwd_raster"] == "rows"
    plain = B.Context(0, raster=B.GP_RASTER_ROWS)
    for k, (it, g) in enumerate(zip(items, meta)):
        ref_img = B.gp_render_slices(plain, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["axis"])
        assert torch.equal(it["out"], ref_img), k
        o = oracle.render(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"], axis=it["axis"])
        assert_forward_close(np32(it["out"]), o, f"batch item {k}")
        og = oracle.render_backward(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"],
                                    it["dL_dI"].cpu().numpy(), axis=it["axis"])
        assert_grads_close(it["grads"], og, f"batch item {k}")
    plan.close()


def test_batch_per_thread_forms_match_plain_calls_and_oracle():
    """A plan of a context with per-thread rasterisers (2 pixels per thread
    forward, 4 backward) runs them over every batch key; images equal the plain
    per-thread calls' bitwise and both passes meet the oracle's parity bars."""
    ctx = B.Context(0, fwd_px=2, bwd_px=4)
    items, meta = _items(seed=12, n=4)
    plan = B.BatchPlan(ctx, items)
    plan.run()
    plan.wait()
    info = plan.info()
    assert (info["fwd_raster"], info["fwd_px"], info["bwd_raster"], info["bwd_px"]) == ("pixels", 2, "pixels", 4)
    plain = B.Context(0, fwd_px=2, bwd_px=4)
    for k, (it, g) in enumerate(zip(items, meta)):
        ref_img = B.gp_render_slices(plain, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["axis"])
        assert torch.equal(it["out"], ref_img), k
        o = oracle.render(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"], axis=it["axis"])
        assert_forward_close(np32(it["out"]), o, f"batch item {k}")
        og = oracle.render_backward(g.mu, g.scale, g.quat, g.alpha, it["z"], it["H"], it["W"], it["sigma_z"],
                                    it["dL_dI"].cpu().numpy(), axis=it["axis"])
        assert_grads_close(it["grads"], og, f"batch item {k}")
    plan.close()
