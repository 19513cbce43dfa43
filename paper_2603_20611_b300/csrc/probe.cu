// probe.cu -- FP32-pipe throughput probe used to measure the ALU roofline
// denominator at the clocks in force (the measured-peak file carries only HBM
// and tensor-core figures).  Each thread runs `iters` iterations of independent
// FMA chains, so the FP32 pipe, not latency, limits the rate.  Three forms:
//   mode 0: 8 scalar FFMA chains               (8 lane FMAs per iteration)
//   mode 1: 8 packed fp32x2 FFMA2 chains       (16 lane FMAs per iteration)
//   mode 2: 4 FFMA2 chains + 8 FFMA chains     (16 lane FMAs per iteration)
//   mode 3: 8 chains x <- 2^-x of the SFU instruction ex2.approx (8 lane
//           exponentials per iteration; x stays in [1/2, 1]): the SFU rate,
//           the denominator of the roofline of the GP_EXP_HW variant
// The packed forms show whether the paired instruction adds FP32 throughput or
// only saves issue slots.
#include <cuda_runtime.h>

#include "gp_common.cuh"
#include "gp_internal.h"

namespace gp {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

template <int MODE>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, float* __restrict__ out) {
  const int tid = blockIdx.x * PROBE_THREADS + threadIdx.x;
  const float m = 0.99993f, c = 7.0e-5f;
  float s = 0.f;
  if constexpr (MODE == 3) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.5f + 1e-3f * (float)((tid + k) & 15);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = exp2_hw(-a[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
  } else if constexpr (MODE == 0) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * (float)((tid + k) & 15);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
  } else {
    constexpr int NP = MODE == 1 ? 8 : 4;  // packed chains
    constexpr int NS = MODE == 1 ? 0 : 8;  // scalar chains
    float2 p[NP];
    float a[NS > 0 ? NS : 1];
#pragma unroll
    for (int k = 0; k < NP; ++k)
      p[k] = make_float2(1.0f + 1e-3f * (float)((tid + k) & 15), 1.0f + 1e-3f * (float)((tid + k + 7) & 15));
#pragma unroll
    for (int k = 0; k < NS; ++k) a[k] = 1.0f + 1e-3f * (float)((tid + k + 3) & 15);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < NP; ++k) p[k] = __ffma2_rn(p[k], m2, c2);
#pragma unroll
      for (int k = 0; k < NS; ++k) a[k] = fmaf(a[k], m, c);
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) s += p[k].x + p[k].y;
#pragma unroll
    for (int k = 0; k < NS; ++k) s += a[k];
  }
  out[tid] = s;
}

int64_t fma_probe_threads(int sm_count) { return (int64_t)sm_count * PROBE_BLOCKS_PER_SM * PROBE_THREADS; }

int fma_probe_lane_fmas(int mode) { return (mode == 0 || mode == 3) ? 8 : 16; }

void launch_fma_probe(int sm_count, int mode, int iters, float* out, cudaStream_t st) {
  const int grid = sm_count * PROBE_BLOCKS_PER_SM;
  if (mode == 1) k_fma_probe<1><<<grid, PROBE_THREADS, 0, st>>>(iters, out);
  else if (mode == 2) k_fma_probe<2><<<grid, PROBE_THREADS, 0, st>>>(iters, out);
  else if (mode == 3) k_fma_probe<3><<<grid, PROBE_THREADS, 0, st>>>(iters, out);
  else k_fma_probe<0><<<grid, PROBE_THREADS, 0, st>>>(iters, out);
  note_launch();
}

}  // namespace gp
