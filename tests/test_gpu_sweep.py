"""A seeded sweep of small random configurations against the FP64 oracle:
set sizes from 1 to 500 Gaussians, images from 1 x 1 to 70 x 70 (never tile
multiples by construction), 1 to 6 planes anywhere in and beyond the volume,
sigma_z from 0.3 to 6, scale modifiers, all three axes and oblique views, both
tile sizes, the three exponentials, both backward modes and both rasteriser
forms (odd cases: row units).

Every case checks the forward and every gradient.  The device culls terms
below eps = 1e-6 of their pair (the culling reading), the oracle culls none,
and every term is >= 0; ``tests/truncation.py`` bounds, per pixel and per
parameter, what the culling may drop.  Where that bound leaves at least half
of each bar free the parity bars apply as they are; elsewhere (images that
show only far tails, or many overlapping tail regions) the device is held to
the oracle minus at most the bound, and the case runs a second time at
eps = 1e-12, where the bound is far inside the bars, under the bars as they
are."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests import truncation
from tests.gpu_util import (FWD_MAX_ABS_FRAC, FWD_REL_L2, GRAD_REL_L2, assert_forward_close,
                            assert_grads_close, dev_set, np32)

pytestmark = pytest.mark.gpu

N_CASES = 64


def _case(k):
    rng = np.random.Generator(np.random.PCG64(9000 + k))
    n = int(rng.integers(1, 501))
    H, W = int(rng.integers(1, 71)), int(rng.integers(1, 71))
    depth = int(rng.integers(4, 40))
    g = synth.small(seed=9100 + k, n=n, extent=(W, H, depth))
    g.scale = (g.scale * np.exp(rng.uniform(-0.7, 1.2))).astype(np.float32)
    S = int(rng.integers(1, 7))
    z = rng.uniform(-3.0, depth + 3.0, S).astype(np.float32)
    cfg = dict(sigma=float(np.exp(rng.uniform(np.log(0.3), np.log(6.0)))),
               mod=float(rng.uniform(0.5, 2.0)),
               tile=int(rng.choice([8, 16])),
               exp=int(rng.choice([B.GP_EXP_POLY, B.GP_EXP_POLY_ROW, B.GP_EXP_HW])),
               det=bool(rng.integers(0, 2)),
               view=int(rng.integers(0, 4)))  # 0-2 axis, 3 oblique
    return g, z, H, W, cfg, rng


def _oblique(rng):
    # a random rotation (QR of a Gaussian matrix) and an offset
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q.astype(np.float32), rng.uniform(-5.0, 5.0, 3).astype(np.float32)


def _run(g, z, H, W, cfg, view, G, eps):
    c = B.Context(0, tile=cfg["tile"], exp_mode=cfg["exp"], deterministic=cfg["det"], eps=eps,
                  raster=cfg["raster"])
    gs = dev_set(g, cfg["mod"])
    Gd = torch.from_numpy(G).cuda()
    if cfg["view"] < 3:
        ax = cfg["view"]
        out = B.gp_render_slices(c, gs, z, H, W, cfg["sigma"], ax)
        grads = B.gp_render_backward(c, gs, z, H, W, cfg["sigma"], Gd, ax)
    else:
        out = B.gp_render_slices(c, gs, z, H, W, cfg["sigma"], view=view)
        grads = B.gp_render_backward(c, gs, z, H, W, cfg["sigma"], Gd, view=view)
    return np32(out), [t.detach().cpu().numpy().astype(np.float64) for t in grads]


def _within_bars(ref, gref, b, gb):
    """True when the culling bound uses at most half of each parity bar."""
    peak = float(np.abs(ref).max())
    fwd = b.max() <= 0.5 * FWD_MAX_ABS_FRAC * peak and \
        np.linalg.norm(b) <= 0.5 * FWD_REL_L2 * np.linalg.norm(ref)
    grad = all(np.linalg.norm(bb) <= 0.5 * GRAD_REL_L2 * np.linalg.norm(r) for bb, r in zip(gb, gref))
    return fwd and grad


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_configuration(k):
    g, z, H, W, cfg, rng = _case(k)
    # odd cases take the row-unit rasterisers, even ones the default forms
    cfg["raster"] = B.GP_RASTER_ROWS if (k % 2 and cfg["exp"] != B.GP_EXP_POLY_ROW) else B.GP_RASTER_AUTO
    o = (g.mu, g.scale, g.quat, g.alpha)
    G = synth.random_field(9200 + k, (len(z), H, W))
    if cfg["view"] < 3:
        view = None
        ref = oracle.render(*o, z, H, W, cfg["sigma"], axis=cfg["view"], scale_mod=cfg["mod"])
        gref = oracle.render_backward(*o, z, H, W, cfg["sigma"], G, axis=cfg["view"], scale_mod=cfg["mod"])
        bview = truncation.axis_view(cfg["view"])
    else:
        view = _oblique(rng)
        ref = oracle.render(*o, z, H, W, cfg["sigma"], scale_mod=cfg["mod"], view=view)
        gref = oracle.render_backward(*o, z, H, W, cfg["sigma"], G, scale_mod=cfg["mod"], view=view)
        bview = view
    what = f"case {k}: n={g.n} {H}x{W} S={len(z)} {cfg}"
    b = truncation.forward_bound(g, z, H, W, cfg["sigma"], cfg["mod"], bview)
    gb = truncation.gradient_bound(g, z, H, W, cfg["sigma"], G, cfg["mod"], bview)
    out, grads = _run(g, z, H, W, cfg, view, G, 1e-6)
    if _within_bars(ref, gref, b, gb):
        assert_forward_close(out, ref, what)
        assert_grads_close(grads, gref, what)
        return
    # the oracle minus at most the culled terms, plus the bars' rounding allowance
    peak = float(np.abs(ref).max())
    tol = FWD_MAX_ABS_FRAC * peak
    assert np.all(out <= ref + tol) and np.all(out >= ref - b - tol), \
        f"{what}: forward outside [oracle - culled bound, oracle] (peak {peak:.3e}, bound {b.max():.3e})"
    assert np.linalg.norm(out - ref) <= np.linalg.norm(b) + FWD_REL_L2 * np.linalg.norm(ref), what
    for name, a, r, bb in zip(("mu", "scale", "quat", "alpha"), grads, gref, gb):
        e = np.linalg.norm(a.reshape(r.shape) - r)
        lim = np.linalg.norm(bb) + GRAD_REL_L2 * np.linalg.norm(r)
        assert e <= lim, f"{what}: d{name} error {e:.3e} > culled bound + bar {lim:.3e}"
    # and under the bars as they are, with a culling bound far inside them
    eps = 1e-12
    b = truncation.forward_bound(g, z, H, W, cfg["sigma"], cfg["mod"], bview, eps=eps)
    gb = truncation.gradient_bound(g, z, H, W, cfg["sigma"], G, cfg["mod"], bview, eps=eps)
    assert _within_bars(ref, gref, b, gb), f"{what}: eps {eps} still leaves the bars"
    out, grads = _run(g, z, H, W, cfg, view, G, eps)
    assert_forward_close(out, ref, what + f" eps {eps}")
    assert_grads_close(grads, gref, what + f" eps {eps}")
