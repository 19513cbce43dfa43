// probe.cu -- FP32-pipe throughput probe used to measure the ALU roofline
// denominator at the clocks in force (the measured-peak file carries only HBM
// and tensor-core figures).  Each thread runs `iters` iterations of eight
// independent FMA chains, so the FP32 pipe, not latency, limits the rate.
#include <cuda_runtime.h>

#include "gp_internal.h"

namespace gp {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, float* __restrict__ out) {
  const int tid = blockIdx.x * PROBE_THREADS + threadIdx.x;
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * (float)((tid + k) & 15);
  const float m = 0.99993f, c = 7.0e-5f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[tid] = s;
}

int64_t fma_probe_threads(int sm_count) { return (int64_t)sm_count * PROBE_BLOCKS_PER_SM * PROBE_THREADS; }

void launch_fma_probe(int sm_count, int iters, float* out, cudaStream_t st) {
  k_fma_probe<<<sm_count * PROBE_BLOCKS_PER_SM, PROBE_THREADS, 0, st>>>(iters, out);
  note_launch();
}

}  // namespace gp
