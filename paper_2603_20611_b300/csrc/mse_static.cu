// mse_static.cu -- gp_mse_grad_noalloc: the MSE loss / gradient without any
// device allocation.
//
// gp_mse_grad keeps its per-block partial sums and the uploaded target slice
// indices in the context's workspace, which grows with cudaMalloc.  Some callers
// cannot allow that: a process whose device memory is already reserved by
// another allocator (a framework's caching allocator or a fixed pool) can see a
// fresh cudaMalloc fail even though memory is free in that pool, and a
// latency-bound serving loop cannot pay for cudaMalloc / cudaFree, which
// synchronise the device.  This variant needs no context and keeps its scratch
// in one file-scope device array of fixed size instead.
//
// The array lives in the library's device module, so every GPU that loads the
// library holds it (about 1.06 MiB) until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress on the first call made on each device, with that
// device current.  Only a successful lookup is kept: after a failed one (for
// example under an error left by earlier work) the next call tries again.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

constexpr int kNoallocPartials = 1 << 18;  // per-block partial sums (floats), 1 MiB
constexpr int kNoallocIndex = 1 << 14;     // target slice indices (ints), 64 KiB
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoallocPartials + kNoallocIndex];

struct NoallocDevice {
  std::mutex mu;
  float* ptr = nullptr;  // set once the lookup has succeeded
};
static NoallocDevice g_noalloc_dev[kNoallocMaxDevices];

// The scratch's device address on the current device `dev`, or nullptr.
static float* noalloc_scratch(int dev) {
  NoallocDevice& d = g_noalloc_dev[dev];
  std::lock_guard<std::mutex> lk(d.mu);
  if (!d.ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) == cudaSuccess)
      d.ptr = (float*)p;
    else
      cudaGetLastError();
  }
  return d.ptr;
}

}  // namespace gp

using namespace gp;

extern "C" GP_API gp_status gp_mse_grad_noalloc(const float* I, const float* T, const int* t_index, int S,
                                                int H, int W, float* dL_dI, float* loss, void* stream) {
  if (S < 0 || H <= 0 || W <= 0) return GP_ERR_ARG;
  if (S == 0) return GP_OK;
  if (!I || !T || !dL_dI) return GP_ERR_ARG;
  const int64_t HW = (int64_t)H * W;
  // sizes beyond the fixed scratch are rejected before anything runs
  if (S > kNoallocPartials) return GP_ERR_OVERFLOW;
  if ((int64_t)mse_tmp_floats(S, HW) > kNoallocPartials) return GP_ERR_OVERFLOW;
  if (t_index && S > kNoallocIndex) return GP_ERR_OVERFLOW;
  if (t_index)
    for (int s = 0; s < S; ++s)
      if (t_index[s] < 0) return GP_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  float* scratch = noalloc_scratch(dev);
  if (!scratch) return GP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int* tid = nullptr;
  if (t_index) {
    int* dst = (int*)(scratch + kNoallocPartials);
    uint32_t* d1[1] = {(uint32_t*)dst};
    const void* s1[1] = {t_index};
    if (put_words(st, 1, d1, s1, &S) != cudaSuccess) {
      cudaGetLastError();
      return GP_ERR_CUDA;
    }
    tid = dst;
  }
  // every partial the final reduction reads is written first by the per-slice
  // kernel of this call, so nothing has to be cleared
  launch_mse(I, T, tid, S, HW, dL_dI, loss, scratch, st);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  return GP_OK;
}
