"""GPU tests of the fit loop's device update (gp_adam_*): each step against the
FP64 oracle's Adam (the paper's rates and schedule, Sec. 5.1) in both
parameterisations, argument checks, and a short render -> MSE -> backward ->
Adam loop whose loss curve must follow the same loop driven by the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import optim
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import dev_set, np32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("act", [True, False])
def test_adam_steps_match_oracle(act):
    ctx = B.Context(0)
    g = synth.small(seed=301, n=3001, extent=(64, 64, 32))
    gs = dev_set(g)
    rng = np.random.Generator(np.random.PCG64(302))
    opt = B.Adam(ctx, gs, total_steps=7, mu_extent=64.0, log_scale_logit_alpha=act)
    ref = optim.FitState(g.mu, g.scale, g.quat, g.alpha, log_scale_logit_alpha=act)
    start = [np.asarray(x, np.float64).copy() for x in ref.params()]
    for t in range(1, 10):  # past total_steps: the rate stays at its final value
        grads = [rng.standard_normal(x.shape).astype(np.float32) * (10.0 ** rng.uniform(-3, 1))
                 for x in (g.mu, g.scale, g.quat, g.alpha)]
        opt.step(gs, [torch.from_numpy(x).cuda() for x in grads])
        want = ref.step(grads, t, total=7, extent=64.0)
        for name, got, w, s0 in zip(optim.GROUPS, (gs.mu, gs.scale, gs.quat, gs.alpha), want, start):
            d_got = np32(got).reshape(w.shape) - s0
            d_want = w - s0
            # compare the accumulated update, relative to its size (fp32 state vs fp64)
            err = np.abs(d_got - d_want).max() / max(np.abs(d_want).max(), 1e-30)
            assert err < 2e-3, (t, name, err)


def test_adam_rejects_bad_arguments():
    ctx = B.Context(0)
    gs = dev_set(synth.small(seed=303, n=16, extent=(8, 8, 8)))
    opt = B.Adam(ctx, gs)
    z = [torch.zeros_like(x) for x in (gs.mu, gs.scale, gs.quat, gs.alpha)]
    opt.t = -1  # the next step would be t = 0
    with pytest.raises(B.GPError):
        opt.step(gs, z)
    opt.t = 0
    opt.cfg.beta2 = 1.0
    with pytest.raises(B.GPError):
        opt.step(gs, z)


def test_fit_loop_follows_the_oracle_loop():
    """Ten steps of the fit loop on a tiny stack (150 Gaussians, 32 x 32, 4 of 8
    planes per step): the GPU loop (fp32) and the oracle loop (fp64 render,
    backward and Adam) see the same targets and slice batches; their loss curves
    must agree, and the loss over the whole stack must fall by the same amount."""
    ctx = B.Context(0, deterministic=True)
    g0 = synth.small(seed=310, n=150, extent=(32, 32, 8))
    tgt = synth.small(seed=311, n=150, extent=(32, 32, 8))
    zs_all = synth.slice_positions(range(8))
    T = oracle.render(tgt.mu, tgt.scale, tgt.quat, tgt.alpha, zs_all, 32, 32, 1.5)
    T_dev = torch.from_numpy(T.astype(np.float32)).cuda()
    gs = dev_set(g0)
    opt = B.Adam(ctx, gs, total_steps=10, mu_extent=32.0, lr_mu=2e-3, lr_alpha=5e-2)
    ref = optim.FitState(g0.mu, g0.scale, g0.quat, g0.alpha)
    gpu_loss, orc_loss = [], []
    for t in range(1, 11):
        idx = synth.slice_batch(320 + t, 8, 8, 4)
        z = zs_all[idx]
        I = B.gp_render_slices(ctx, gs, z, 32, 32, 1.5)
        loss = torch.zeros(1, device="cuda")
        dL, _ = B.gp_mse_grad(ctx, I, T_dev, t_index=idx, loss=loss)
        grads = B.gp_render_backward(ctx, gs, z, 32, 32, 1.5, dL)
        opt.step(gs, grads)
        gpu_loss.append(loss.item())
        mu, s, q, a = ref.params()
        Io = oracle.render(mu, s, q, a, z, 32, 32, 1.5)
        L, dLo = oracle.mse(Io, T[idx])
        go = oracle.render_backward(mu, s, q, a, z, 32, 32, 1.5, dLo)
        ref.step(go, t, lrs=dict(optim.PAPER_LR, mu=2e-3, alpha=5e-2), total=10, extent=32.0)
        orc_loss.append(L)
    np.testing.assert_allclose(gpu_loss, orc_loss, rtol=2e-3)
    # the loss over the whole 8-plane stack fell, for both loops, by the same amount
    full0 = oracle.mse(oracle.render(g0.mu, g0.scale, g0.quat, g0.alpha, zs_all, 32, 32, 1.5), T)[0]
    full_orc = oracle.mse(oracle.render(*ref.params(), zs_all, 32, 32, 1.5), T)[0]
    full_gpu = oracle.mse(oracle.render(np32(gs.mu), np32(gs.scale), np32(gs.quat), np32(gs.alpha), zs_all, 32,
                                        32, 1.5), T)[0]
    assert full_orc < 0.95 * full0
    assert full_gpu == pytest.approx(full_orc, rel=2e-3)
