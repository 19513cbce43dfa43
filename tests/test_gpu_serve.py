"""GPU tests of the serving loop: each result is the same alone and in a mix of
concurrent, batched requests; slice results equal the plain render (and the
oracle); admission holds requests back under a small memory budget; bad
requests are rejected at submit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, dev_set, np32

pytestmark = pytest.mark.gpu


def _sets():
    a = synth.small(seed=71, n=3000, extent=(96, 96, 48))
    b = synth.small(seed=72, n=1500, extent=(96, 96, 48))
    return [a, b]


def _requests(rng, n):
    reqs = []
    for _ in range(n):
        kind = int(rng.choice([B.GP_REQ_SLICE, B.GP_REQ_STACK, B.GP_REQ_VOXELIZE], p=[0.5, 0.3, 0.2]))
        sid = int(rng.integers(0, 2))
        if kind == B.GP_REQ_VOXELIZE:
            reqs.append(dict(kind=kind, set_id=sid, X=40, Y=36, Z=24, shape=(24, 36, 40)))
        else:
            S = 1 if kind == B.GP_REQ_SLICE else int(rng.integers(2, 6))
            z = rng.uniform(0, 48, S).astype(np.float32)
            reqs.append(dict(kind=kind, set_id=sid, z=z, H=96, W=96, sigma_z=2.0, axis=2, shape=(S, 96, 96)))
    return reqs


def _submit(srv, r, out):
    if r["kind"] == B.GP_REQ_VOXELIZE:
        return srv.submit(r["kind"], r["set_id"], out, X=r["X"], Y=r["Y"], Z=r["Z"])
    return srv.submit(r["kind"], r["set_id"], out, z=r["z"], H=r["H"], W=r["W"], sigma_z=r["sigma_z"],
                      axis=r["axis"])


def _wait(srv, t):
    for _ in range(600):
        res = srv.poll(t, timeout_ms=100)
        if res is not None:
            return res
    raise AssertionError("request did not complete")


def _long_stacks(srv, n, sid, planes):
    """n stacks of `planes` planes of 1024^2 of a 500k-Gaussian set (several ms each)."""
    z = (np.arange(planes, dtype=np.float32) * 4.0 + 0.5)
    outs = [torch.empty(planes, 1024, 1024, device="cuda") for _ in range(n)]
    return [srv.submit(B.GP_REQ_STACK, sid, o, z=z, H=1024, W=1024, sigma_z=3.0) for o in outs], outs


def test_results_alone_equal_results_in_the_mix():
    ctx = B.Context(0)
    sets = [dev_set(g) for g in _sets()]
    big = dev_set(synth.microscopy(seed=1002, n=500_000, extent=(1024, 1024, 256)))
    rng = np.random.Generator(np.random.PCG64(5))
    reqs = _requests(rng, 24)
    srv = B.Server(ctx, workers=3, max_batch_slices=32)
    ids = [srv.load_set(g) for g in sets]
    assert ids == [0, 1]
    big_id = srv.load_set(big)
    alone = []
    for r in reqs:
        out = torch.full(r["shape"], float("nan"), device="cuda")
        res = _wait(srv, _submit(srv, r, out))
        assert res["status"] == B.GP_OK and res["batch_size"] == 1
        alone.append(out)
    # three long stacks occupy the three workers while the mix is queued behind
    # them, so the mix is taken in batches and runs concurrently on the workers
    long_t, _ = _long_stacks(srv, 3, big_id, 32)
    outs = [torch.full(r["shape"], float("nan"), device="cuda") for r in reqs]
    tickets = [_submit(srv, r, o) for r, o in zip(reqs, outs)]
    results = [_wait(srv, t) for t in tickets]
    assert all(_wait(srv, t)["status"] == B.GP_OK for t in long_t)
    assert all(res["status"] == B.GP_OK for res in results)
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
    assert max(res["batch_size"] for res in results) > 1, "the mix was never batched"
    st = srv.stats()
    assert st["max_inflight_requests"] > 1, "requests never overlapped"
    assert st["batches"] < st["completed"]
    assert st["completed"] == 2 * len(reqs) + len(long_t) and st["failed"] == 0
    srv.close()


def test_voxelize_requests_of_one_set_and_grid_are_batched():
    ctx = B.Context(0)
    a, b = [dev_set(g) for g in _sets()]
    big = dev_set(synth.microscopy(seed=1002, n=500_000, extent=(1024, 1024, 256)))
    srv = B.Server(ctx, workers=1, max_batch_slices=64)
    ia, ib, ibig = srv.load_set(a), srv.load_set(b), srv.load_set(big)
    long_t, _ = _long_stacks(srv, 2, ibig, 64)  # the worker is busy while the rest queue up
    same = [torch.full((24, 36, 40), float("nan"), device="cuda") for _ in range(5)]
    t_same = [srv.submit(B.GP_REQ_VOXELIZE, ia, o, X=40, Y=36, Z=24) for o in same]
    other_grid = torch.full((24, 36, 48), float("nan"), device="cuda")
    other_set = torch.full((24, 36, 40), float("nan"), device="cuda")
    t_grid = srv.submit(B.GP_REQ_VOXELIZE, ia, other_grid, X=48, Y=36, Z=24)
    t_set = srv.submit(B.GP_REQ_VOXELIZE, ib, other_set, X=40, Y=36, Z=24)
    res = [_wait(srv, t) for t in t_same]
    r_grid, r_set = _wait(srv, t_grid), _wait(srv, t_set)
    assert all(_wait(srv, t)["status"] == B.GP_OK for t in long_t)
    assert all(r["status"] == B.GP_OK for r in res + [r_grid, r_set])
    assert [r["batch_size"] for r in res] == [5] * 5
    assert r_grid["batch_size"] == 1 and r_set["batch_size"] == 1
    ref = B.gp_voxelize(ctx, a, 40, 36, 24)
    for o in same:
        assert torch.equal(o, ref)
    assert torch.equal(other_grid, B.gp_voxelize(ctx, a, 48, 36, 24))
    assert torch.equal(other_set, B.gp_voxelize(ctx, b, 40, 36, 24))
    srv.close()


def test_loading_sets_while_requests_run():
    """Registering sets grows the server's set table while workers render
    requests of earlier sets: every result is still right."""
    import threading
    ctx = B.Context(0)
    g = _sets()[0]
    gs = dev_set(g)
    srv = B.Server(ctx, workers=3, max_batch_slices=8)
    sid = srv.load_set(gs)
    rng = np.random.Generator(np.random.PCG64(8))
    zs = [rng.uniform(0, 48, int(rng.integers(1, 4))).astype(np.float32) for _ in range(60)]
    outs = [torch.full((len(z), 96, 96), float("nan"), device="cuda") for z in zs]
    extra = [dev_set(synth.small(seed=300 + k, n=10, extent=(16, 16, 8))) for k in range(4)]
    loaded = []

    def loader():
        for k in range(400):
            loaded.append(srv.load_set(extra[k % 4]))

    th = threading.Thread(target=loader)
    th.start()
    tickets = [srv.submit(B.GP_REQ_STACK, sid, o, z=z, H=96, W=96, sigma_z=2.0) for z, o in zip(zs, outs)]
    th.join()
    assert all(_wait(srv, t)["status"] == B.GP_OK for t in tickets)
    assert sorted(loaded) == list(range(1, 401))
    for z, o in zip(zs, outs):
        assert torch.equal(o, B.gp_render_slices(ctx, gs, z, 96, 96, 2.0))
    srv.close()


def test_batched_slices_match_plain_render_and_oracle():
    ctx = B.Context(0)
    g = _sets()[0]
    gs = dev_set(g)
    srv = B.Server(ctx, workers=1, max_batch_slices=64)
    sid = srv.load_set(gs)
    rng = np.random.Generator(np.random.PCG64(6))
    zs = [rng.uniform(0, 48, 1).astype(np.float32) for _ in range(12)]
    outs = [torch.empty(1, 96, 96, device="cuda") for _ in zs]
    tickets = [srv.submit(B.GP_REQ_SLICE, sid, o, z=z, H=96, W=96, sigma_z=2.0) for z, o in zip(zs, outs)]
    res = [_wait(srv, t) for t in tickets]
    assert max(r["batch_size"] for r in res) > 1  # queued slices were rendered together
    for z, o in zip(zs, outs):
        ref = B.gp_render_slices(ctx, gs, z, 96, 96, 2.0)
        assert torch.equal(o, ref)
    z_all = np.concatenate(zs)
    ref = oracle.render(g.mu, g.scale, g.quat, g.alpha, z_all, 96, 96, 2.0)
    assert_forward_close(np.concatenate([np32(o) for o in outs]), ref, "served slices")
    srv.close()


def test_admission_under_a_small_budget():
    ctx = B.Context(0)
    sets = [dev_set(g) for g in _sets()]
    srv = B.Server(ctx, workers=4, hbm_budget_bytes=1)  # only one request in flight at a time
    for g in sets:
        srv.load_set(g)
    rng = np.random.Generator(np.random.PCG64(7))
    reqs = _requests(rng, 12)
    outs = [torch.empty(r["shape"], device="cuda") for r in reqs]
    tickets = [_submit(srv, r, o) for r, o in zip(reqs, outs)]
    results = [_wait(srv, t) for t in tickets]
    assert all(r["status"] == B.GP_OK for r in results)
    st = srv.stats()
    assert st["max_inflight_requests"] == 1 and st["inflight_requests"] == 0
    for r, o in zip(reqs, outs):  # and the results are right
        if r["kind"] != B.GP_REQ_VOXELIZE:
            ref = B.gp_render_slices(ctx, sets[r["set_id"]], r["z"], r["H"], r["W"], r["sigma_z"], r["axis"])
            assert torch.equal(o, ref)
    srv.close()


def test_bad_requests_are_rejected():
    ctx = B.Context(0)
    srv = B.Server(ctx, workers=1)
    sid = srv.load_set(dev_set(_sets()[1]))
    out = torch.empty(1, 8, 8, device="cuda")
    z = np.array([3.0], np.float32)
    for kw in (dict(set_id=5), dict(H=0), dict(sigma_z=0.0), dict(axis=4)):
        a = dict(set_id=sid, H=8, W=8, sigma_z=1.0, axis=2)
        a.update(kw)
        with pytest.raises(B.GPError) as ei:
            srv.submit(B.GP_REQ_SLICE, a["set_id"], out, z=z, H=a["H"], W=a["W"], sigma_z=a["sigma_z"],
                       axis=a["axis"])
        assert ei.value.status == B.GP_ERR_ARG
    with pytest.raises(B.GPError):
        srv.submit(B.GP_REQ_SLICE, sid, out, z=np.array([1.0, 2.0], np.float32), H=8, W=8)  # SLICE needs S == 1
    with pytest.raises(B.GPError):
        srv.poll(12345)
    srv.close()


def _busy_server(ctx, n_long=3):
    """One worker and a 1-byte budget, so requests run one at a time, and n_long
    stacks of a 500k-Gaussian set in front (each several milliseconds): whatever
    is submitted next waits in the queue behind them."""
    g = synth.microscopy(seed=1002, n=500_000, extent=(1024, 1024, 256))
    gs = dev_set(g)
    srv = B.Server(ctx, workers=1, hbm_budget_bytes=1)
    sid = srv.load_set(gs)
    z = (np.arange(64, dtype=np.float32) * 4.0 + 0.5)
    outs = [torch.empty(64, 1024, 1024, device="cuda") for _ in range(n_long)]
    long_t = [srv.submit(B.GP_REQ_STACK, sid, o, z=z, H=1024, W=1024, sigma_z=3.0) for o in outs]
    return srv, sid, gs, long_t, outs


def test_cancel_and_queue_deadline():
    ctx = B.Context(0)
    srv, sid, gs, long_t, _ = _busy_server(ctx)
    out = torch.full((1, 64, 64), float("nan"), device="cuda")
    z = np.array([10.5], np.float32)
    t_cancel = srv.submit(B.GP_REQ_SLICE, sid, torch.empty(1, 64, 64, device="cuda"), z=z, H=64, W=64, sigma_z=3.0)
    srv.cancel(t_cancel)  # still queued behind the long stacks
    t_late = srv.submit(B.GP_REQ_SLICE, sid, torch.empty(1, 64, 64, device="cuda"), z=z, H=64, W=64, sigma_z=3.0,
                        timeout_ms=2.0)
    t_ok = srv.submit(B.GP_REQ_SLICE, sid, out, z=z, H=64, W=64, sigma_z=3.0, timeout_ms=60_000.0)
    assert _wait(srv, t_cancel)["status"] == B.GP_ERR_CANCELLED
    assert _wait(srv, t_late)["status"] == B.GP_ERR_TIMEOUT
    assert _wait(srv, t_ok)["status"] == B.GP_OK
    assert all(_wait(srv, t)["status"] == B.GP_OK for t in long_t)
    assert torch.equal(out, B.gp_render_slices(ctx, gs, z, 64, 64, 3.0))  # the request behind them is right
    # a finished request cannot be cancelled, an unknown ticket is an argument error
    with pytest.raises(B.GPError) as ei:
        srv.cancel(t_ok)
    assert ei.value.status == B.GP_ERR_STATE
    with pytest.raises(B.GPError) as ei:
        srv.cancel(10 ** 9)
    assert ei.value.status == B.GP_ERR_ARG
    st = srv.stats()
    assert st["cancelled"] == 1 and st["expired"] == 1 and st["failed"] == 2 and st["pending"] == 0
    assert st["completed"] == len(long_t) + 3
    with pytest.raises(B.GPError) as ei:  # a negative deadline is rejected at submit
        srv.submit(B.GP_REQ_SLICE, sid, out, z=z, H=64, W=64, sigma_z=3.0, timeout_ms=-1.0)
    assert ei.value.status == B.GP_ERR_ARG
    srv.close()


def test_workspace_limit_reports_oom_and_leaves_the_context_usable():
    """A call whose scratch would pass the context's workspace limit fails with
    GP_ERR_OOM and frees the context's workspace; smaller calls on the same
    context still run and are right."""
    g = synth.small(seed=74, n=3000, extent=(96, 96, 48))
    gs = dev_set(g)
    z = synth.slice_positions(range(8))
    free = B.Context(0)
    ref = B.gp_render_slices(free, gs, z, 96, 96, 2.0)
    need = free.workspace_bytes()
    assert need > 0
    ctx = B.Context(0, workspace_limit=need // 4)
    with pytest.raises(B.GPError) as ei:
        B.gp_render_slices(ctx, gs, z, 96, 96, 2.0)
    assert ei.value.status == B.GP_ERR_OOM and "workspace limit" in str(ei.value)
    assert ctx.workspace_bytes() == 0
    small = dev_set(synth.small(seed=75, n=20, extent=(16, 16, 8)))
    zs = synth.slice_positions(range(2))
    got = B.gp_render_slices(ctx, small, zs, 16, 16, 2.0)
    assert torch.equal(got, B.gp_render_slices(free, small, zs, 16, 16, 2.0))
    big = B.Context(0, workspace_limit=4 * need)
    assert torch.equal(B.gp_render_slices(big, gs, z, 96, 96, 2.0), ref)
