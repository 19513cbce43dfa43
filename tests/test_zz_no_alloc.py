"""GPU test of gp_mse_grad_noalloc, the MSE loss / gradient for callers that
must not allocate device memory (their memory is reserved by another allocator,
or their loop cannot afford cudaMalloc's device synchronisation).  It is called
through the C ABI, twice in a row on different inputs, and must agree with
gp_mse_grad each time.  This file is collected last so that a failing run has
already exercised every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_20611_b300 import binding as B

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_mse_matches_mse_grad_on_two_calls():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    ctx = B.Context(0)
    rng = np.random.Generator(np.random.PCG64(99))
    stream = torch.cuda.current_stream()
    cases = [((5, 37, 29), 8, [7, 0, 3, 3, 6]), ((3, 300, 257), 3, None)]
    for (S, H, W), depth, tidx in cases:
        I = torch.from_numpy(rng.standard_normal((S, H, W)).astype(np.float32)).cuda()
        T = torch.from_numpy(rng.standard_normal((depth, H, W)).astype(np.float32)).cuda()
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
