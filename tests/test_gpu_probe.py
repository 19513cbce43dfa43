"""GPU tests of the throughput probes behind the roofline denominators: every
mode computes what its chains define (so the timed work is really done), and
bad arguments are refused."""
import numpy as np
import pytest
import torch

from paper_2603_20611_b300 import binding as B

pytestmark = pytest.mark.gpu


def _chain_fma(a0, m, c, n):
    # closed form of a <- a m + c after n steps
    return m ** n * a0 + c * (1.0 - m ** n) / (1.0 - m)


def test_fma_modes_compute_their_chains():
    ctx = B.Context(0)
    n_thr = int(B.lib.gp_fma_probe_threads(ctx.h))
    iters = 300
    m, c = 0.99993, 7.0e-5
    tid = np.arange(n_thr)
    for mode, lanes in ((0, 8), (1, 16), (2, 16)):
        out, ops = ctx.fma_probe(iters, mode=mode)
        torch.cuda.synchronize()
        assert ops == n_thr * iters * lanes
        got = out.cpu().numpy().astype(np.float64)
        if mode == 0:
            want = sum(_chain_fma(1.0 + 1e-3 * ((tid + k) & 15), m, c, iters) for k in range(8))
        elif mode == 1:
            want = sum(_chain_fma(1.0 + 1e-3 * ((tid + k) & 15), m, c, iters) +
                       _chain_fma(1.0 + 1e-3 * ((tid + k + 7) & 15), m, c, iters) for k in range(8))
        else:
            want = (sum(_chain_fma(1.0 + 1e-3 * ((tid + k) & 15), m, c, iters) +
                        _chain_fma(1.0 + 1e-3 * ((tid + k + 7) & 15), m, c, iters) for k in range(4)) +
                    sum(_chain_fma(1.0 + 1e-3 * ((tid + k + 3) & 15), m, c, iters) for k in range(8)))
        np.testing.assert_allclose(got, want, rtol=1e-4)


def test_sfu_mode_reaches_the_fixed_point_of_two_to_the_minus_x():
    ctx = B.Context(0)
    n_thr = int(B.lib.gp_fma_probe_threads(ctx.h))
    out, ops = ctx.fma_probe(200, mode=3)
    torch.cuda.synchronize()
    assert ops == n_thr * 200 * 8
    # x = 2^-x at x* = W(ln 2) / ln 2; the iteration contracts (|d/dx 2^-x| = x* ln 2 < 1/2)
    xs = 0.5
    for _ in range(200):
        xs = 2.0 ** -xs
    assert abs(xs - 2.0 ** -xs) < 1e-12
    np.testing.assert_allclose(out.cpu().numpy() / 8.0, xs, rtol=1e-5)


def test_bad_probe_arguments():
    ctx = B.Context(0)
    out = torch.empty(int(B.lib.gp_fma_probe_threads(ctx.h)), device="cuda")
    for mode, iters in ((4, 10), (-1, 10), (0, 0)):
        with pytest.raises(B.GPError) as ei:
            ctx.fma_probe(iters, out=out, mode=mode)
        assert ei.value.status == B.GP_ERR_ARG
    assert B.lib.gp_fma_probe_lane_fmas(4) == 0 and B.lib.gp_fma_probe_lane_fmas(3) == 8
