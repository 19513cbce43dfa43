"""GPU parity of the paper's photometric loss L = L1 + lambda (1 - SSIM)
(Eq. 11, gp_l1_dssim_grad) with the FP64 oracle: loss terms and dL/dI on
ragged stacks (image sides not multiples of the 32-pixel tile, borders with
zero-padded windows), target slices chosen by index, rendered inputs, a
full-size 1024^2 pair of slices, and argument checks."""
import numpy as np
import pytest
import torch

import oracle
from oracle import loss as orc_loss
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import GRAD_REL_L2, dev_set, np32, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _pair(seed, shape, noise=0.1):
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.uniform(0, 1, shape).astype(np.float32)
    I = np.clip(T + noise * rng.standard_normal(shape), 0, 1).astype(np.float32)
    return I, T


def _check(ctx, I, T, lam=0.2, t_index=None):
    Id, Td = torch.from_numpy(I).cuda(), torch.from_numpy(T).cuda()
    out = torch.zeros(3, device="cuda")
    g, _ = B.gp_l1_dssim_grad(ctx, Id, Td, t_index=t_index, lam=lam, loss=out)
    Tsel = T if t_index is None else T[np.asarray(t_index)]
    L, L1, ms, gref = orc_loss.l1_dssim(I.astype(np.float64), Tsel.astype(np.float64), lam)
    got = out.cpu().numpy().astype(np.float64)
    # sums of fp32 terms taken in double; SSIM's variances lose ~1e-7 x mean^2 / var
    assert got[1] == pytest.approx(L1, rel=1e-6)
    assert got[2] == pytest.approx(ms, rel=2e-6, abs=2e-6)
    assert got[0] == pytest.approx(L, rel=2e-6, abs=1e-6)
    e = rel_l2(np32(g), gref)
    assert e <= GRAD_REL_L2, e
    return e


@pytest.mark.parametrize("S,H,W", [(1, 32, 32), (3, 45, 70), (2, 33, 33), (1, 100, 7), (2, 5, 64)])
def test_loss_matches_oracle_on_ragged_stacks(ctx, S, H, W):
    I, T = _pair(S * 1000 + H * 10 + W, (S, H, W))
    _check(ctx, I, T)


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_weights(ctx, lam):
    I, T = _pair(7, (2, 40, 50), 0.3)
    _check(ctx, I, T, lam=lam)


def test_target_slices_by_index(ctx):
    I, _ = _pair(8, (3, 48, 40))
    _, T = _pair(9, (6, 48, 40))
    _check(ctx, I, T, t_index=[4, 0, 4])


def test_rendered_slices_against_rendered_target(ctx):
    g = synth.small(seed=11, n=1500, extent=(64, 64, 16))
    tg = synth.small(seed=12, n=1500, extent=(64, 64, 16))
    z = synth.slice_positions([1, 6, 11])
    I = B.gp_render_slices(ctx, dev_set(g), z, 64, 64, 2.0)
    T = oracle.render(tg.mu, tg.scale, tg.quat, tg.alpha, z, 64, 64, 2.0).astype(np.float32)
    _check(ctx, I.cpu().numpy(), T)


def test_full_size_pair_of_slices(ctx):
    I, T = _pair(13, (2, 1024, 1024), 0.05)
    _check(ctx, I, T)


def test_identical_images_have_zero_loss_and_gradient(ctx):
    I, _ = _pair(14, (2, 37, 29))
    Id = torch.from_numpy(I).cuda()
    out = torch.zeros(3, device="cuda")
    g, _ = B.gp_l1_dssim_grad(ctx, Id, Id.clone(), loss=out)
    L, L1, ms = out.cpu().numpy()
    assert L1 == 0.0 and abs(ms - 1.0) < 1e-6 and abs(L) < 1e-6
    assert g.abs().max().item() < 1e-9


def test_staging_paths_agree_bitwise(ctx):
    """The stencil passes stage their halo rows as aligned float4 when the width
    is a multiple of 4 and every plane is 16-byte aligned, else pixel by pixel.
    Planes offset by one float take the second path; both must give the same
    bits (the arithmetic after staging is the same)."""
    I, T = _pair(15, (3, 40, 64))
    Ia, Ta = torch.from_numpy(I).cuda(), torch.from_numpy(T).cuda()
    bufI = torch.empty(I.size + 1, device="cuda")
    bufT = torch.empty(T.size + 1, device="cuda")
    Im, Tm = bufI[1:].view(I.shape), bufT[1:].view(T.shape)  # 4 bytes past a 16-byte boundary
    Im.copy_(Ia)
    Tm.copy_(Ta)
    assert Im.data_ptr() % 16 == 4 and Im.is_contiguous()
    la, lm = torch.zeros(3, device="cuda"), torch.zeros(3, device="cuda")
    ga, _ = B.gp_l1_dssim_grad(ctx, Ia, Ta, loss=la)
    gm, _ = B.gp_l1_dssim_grad(ctx, Im, Tm, loss=lm)
    assert torch.equal(ga, gm) and torch.equal(la, lm)
    _check(ctx, I, T)  # and the aligned path against the oracle


def test_bad_arguments(ctx):
    I = torch.zeros(1, 8, 8, device="cuda")
    with pytest.raises(B.GPError):
        B.gp_l1_dssim_grad(ctx, I, I, lam=-0.5)
    with pytest.raises(B.GPError):
        B.gp_l1_dssim_grad(ctx, I, I, lam=float("nan"))
    with pytest.raises(ValueError):
        B.gp_l1_dssim_grad(ctx, I, I, t_index=[3])
