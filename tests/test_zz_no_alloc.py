"""GPU test of gp_mse_grad_noalloc, the MSE loss / gradient for callers that
must not allocate device memory (their memory is reserved by another allocator,
or their loop cannot afford cudaMalloc's device synchronisation).  It is called
through the C ABI, twice in a row on different inputs, and must agree with
gp_mse_grad and with the FP64 oracle's MSE each time; the binding's wrapper
and a call without a loss output are exercised too.  This file is collected
last so that a failing run has already exercised every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2603_20611_b300 import binding as B

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs(rng, S, H, W, depth):
    I = rng.standard_normal((S, H, W)).astype(np.float32)
    T = rng.standard_normal((depth, H, W)).astype(np.float32)
    return I, T


def test_noalloc_mse_matches_mse_grad_and_oracle_on_two_calls():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    ctx = B.Context(0)
    rng = np.random.Generator(np.random.PCG64(99))
    stream = torch.cuda.current_stream()
    cases = [((5, 37, 29), 8, [7, 0, 3, 3, 6]), ((3, 300, 257), 3, None)]
    for (S, H, W), depth, tidx in cases:
        In, Tn = _inputs(rng, S, H, W, depth)
        I, T = torch.from_numpy(In).cuda(), torch.from_numpy(Tn).cuda()
        ref_g = torch.empty_like(I)
        ref_loss = torch.zeros(1, device="cuda")
        B.gp_mse_grad(ctx, I, T, tidx, dL_dI=ref_g, loss=ref_loss)
        got_g = torch.full_like(I, float("nan"))
        got_loss = torch.full((1,), float("nan"), device="cuda")
        ti = None if tidx is None else np.asarray(tidx, np.int32)
        st = B.lib.gp_mse_grad_noalloc(_ptr(I), _ptr(T),
                                       None if ti is None else ti.ctypes.data_as(ctypes.c_void_p),
                                       S, H, W, _ptr(got_g), _ptr(got_loss), ctypes.c_void_p(stream.cuda_stream))
        assert st == B.GP_OK
        torch.cuda.synchronize()
        assert torch.allclose(got_g, ref_g, rtol=1e-6, atol=0.0)
        assert got_loss.item() == pytest.approx(ref_loss.item(), rel=1e-6)
        # and the FP64 oracle's loss and gradient
        L, G = oracle.mse(In, Tn if tidx is None else Tn[tidx])
        np.testing.assert_allclose(got_g.cpu().numpy().astype(np.float64), G, rtol=1e-6, atol=1e-12)
        assert got_loss.item() == pytest.approx(L, rel=1e-5)


def test_noalloc_mse_without_loss_output_and_through_the_binding():
    rng = np.random.Generator(np.random.PCG64(98))
    In, Tn = _inputs(rng, 4, 70, 45, 6)
    I, T = torch.from_numpy(In).cuda(), torch.from_numpy(Tn).cuda()
    tidx = [5, 1, 1, 0]
    L, G = oracle.mse(In, Tn[tidx])
    # loss = NULL: only dL/dI is written
    g0 = torch.full_like(I, float("nan"))
    st = B.lib.gp_mse_grad_noalloc(_ptr(I), _ptr(T), np.asarray(tidx, np.int32).ctypes.data_as(ctypes.c_void_p),
                                   4, 70, 45, _ptr(g0), None, None)
    assert st == B.GP_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(g0.cpu().numpy().astype(np.float64), G, rtol=1e-6, atol=1e-12)
    # the binding's wrapper, on the current torch stream
    loss = torch.zeros(1, device="cuda")
    g1, _ = B.gp_mse_grad_noalloc(I, T, tidx, loss=loss)
    torch.cuda.synchronize()
    assert torch.equal(g1, g0)
    assert loss.item() == pytest.approx(L, rel=1e-5)
    g2, none = B.gp_mse_grad_noalloc(I, T[tidx])
    assert none is None and torch.equal(g2, g0)


def test_noalloc_mse_rejects_sizes_beyond_its_scratch():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    I = torch.zeros(1, 4, 4, device="cuda")
    big = np.zeros(20000, np.int32)
    # rejected on the host before any launch: S exceeds the index capacity
    st = B.lib.gp_mse_grad_noalloc(_ptr(I), _ptr(I), big.ctypes.data_as(ctypes.c_void_p), 20000, 4, 4,
                                   _ptr(I), None, None)
    assert st == B.GP_ERR_OVERFLOW
    # more per-block partial sums than the scratch holds (300 slices x 4096 blocks)
    st = B.lib.gp_mse_grad_noalloc(_ptr(I), _ptr(I), None, 300, 4096, 4096, _ptr(I), None, None)
    assert st == B.GP_ERR_OVERFLOW
    assert B.lib.gp_mse_grad_noalloc(None, None, None, 1, 4, 4, None, None, None) == B.GP_ERR_ARG
