// ssim.cu -- the photometric loss L = L1 + lambda (1 - SSIM) of Eq. 11 and its
// gradient with respect to the rendered slices, sm_103a.
//
// SSIM per slice with an 11 x 11 Gaussian window (sigma 1.5), C1 = 0.01^2,
// C2 = 0.03^2, zero padding at the borders.  With the window moments
// m_I = G*I, m_T = G*T, m_II = G*I^2, m_TT = G*T^2, m_IT = G*(I T):
//   S = (2 m_I m_T + C1)(2 s_IT + C2) / ((m_I^2 + m_T^2 + C1)(s_II + s_TT + C2)),
//   s_II = m_II - m_I^2, s_TT = m_TT - m_T^2, s_IT = m_IT - m_I m_T,
// and, the window being symmetric,
//   d mean(S) / dI = (1/n) [G*(dS/dm_I) + 2 I G*(dS/dm_II) + T G*(dS/dm_IT)].
//
// Two tiled stencil passes over 32 x 32 output tiles with a 5-pixel halo held in
// shared memory, each a separable window sum (11 taps along rows, then 11 along
// columns):
//   K-ssim-stats  the five moments -> S, the three derivatives dS/dm_* (global),
//                 per-block sums of S and |I - T| (double, fixed-order final sum)
//   K-ssim-grad   the window sums of the three derivatives -> dL/dI
// The window sums take two maps per packed fp32x2 instruction ((m_I, m_T) and
// (m_II, m_TT) in the stats pass, (dS/dm_I, dS/dm_II) in the gradient pass),
// rows of the halo are staged as aligned float4 when the width allows, and the
// loss sums stay in fp32 per thread and warp (the SM's FP64 rate is a small
// fraction of its FP32 rate), in double across the warps and blocks.
// About 44 bytes of HBM traffic per pixel in all.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gp_internal.h"

namespace gp {

namespace {

constexpr int kTS = 32;              // output tile side
constexpr int kHalo = 5;             // window radius
constexpr int kWS = kTS + 2 * kHalo; // staged window side (42)
constexpr int kThreads = 256;
static_assert(kTS * (kTS / 4) == kThreads, "one vertical output group of 4 pixels per thread");

struct SsimArgs {
  float w[11];  // 1-D window, normalised to sum 1
  int S, H, W;
  float c1, c2, inv_n, lam;
};

__device__ __forceinline__ bool in_img(const SsimArgs& p, int y, int x) {
  return y >= 0 && y < p.H && x >= 0 && x < p.W;
}

// Stages the kWS x kWS window of N planes around the tile at (x0, y0), zero
// outside the image: store(r, c, v) with window row r and column c (pixel
// (y0 - kHalo + r, x0 - kHalo + c)) and v[n] the pixel of plane n.  With vec
// (W a multiple of 4 and every plane 16-byte aligned) a row is read as 12
// aligned float4 from x0 - 8, which cover the window's columns x0 - 5 ..
// x0 + 36 (a float4 lies wholly inside or wholly outside the image);
// otherwise pixel by pixel.
template <int N, typename Store>
__device__ __forceinline__ void stage_window(const SsimArgs& p, const float* const (&src)[N], int x0, int y0,
                                             bool vec, Store store) {
  // every load of the thread first, then the stores (a store between two
  // loads would hold the second back until the first has landed)
  if (vec) {
    constexpr int NI = (kWS * 12 + kThreads - 1) / kThreads;
    float4 v[NI][N];
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      const int i = threadIdx.x + j * kThreads;
      const int r = i / 12, q = i - r * 12;
      const int y = y0 - kHalo + r, xq = x0 - 8 + 4 * q;
      const bool in = i < kWS * 12 && y >= 0 && y < p.H && xq >= 0 && xq < p.W;
#pragma unroll
      for (int n = 0; n < N; ++n)
        v[j][n] = in ? *reinterpret_cast<const float4*>(src[n] + (int64_t)y * p.W + xq) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      const int i = threadIdx.x + j * kThreads;
      if (i >= kWS * 12) break;
      const int r = i / 12, q = i - r * 12;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = 4 * q + k - 3;  // x = xq + k = x0 - kHalo + c
        if (c < 0 || c >= kWS) continue;
        float e[N];
#pragma unroll
        for (int n = 0; n < N; ++n) e[n] = k == 0 ? v[j][n].x : k == 1 ? v[j][n].y : k == 2 ? v[j][n].z : v[j][n].w;
        store(r, c, e);
      }
    }
  } else {
    constexpr int NI = (kWS * kWS + kThreads - 1) / kThreads;
    float e[NI][N];
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      const int i = threadIdx.x + j * kThreads;
      const int r = i / kWS, c = i - r * kWS;
      const int y = y0 - kHalo + r, x = x0 - kHalo + c;
      const bool in = i < kWS * kWS && in_img(p, y, x);
#pragma unroll
      for (int n = 0; n < N; ++n) e[j][n] = in ? src[n][(int64_t)y * p.W + x] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      const int i = threadIdx.x + j * kThreads;
      if (i >= kWS * kWS) break;
      const int r = i / kWS, c = i - r * kWS;
      store(r, c, e[j]);
    }
  }
}

// 16-byte alignment of every plane a vectorised staging reads.
template <int N>
__device__ __forceinline__ bool planes_aligned(const SsimArgs& p, const float* const (&src)[N]) {
  uintptr_t a = 0;
#pragma unroll
  for (int n = 0; n < N; ++n) a |= reinterpret_cast<uintptr_t>(src[n]);
  return (p.W & 3) == 0 && (a & 15u) == 0;
}

__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

__global__ void __launch_bounds__(kThreads, 5) k_ssim_stats(SsimArgs p, const float* __restrict__ I,
                                                        const float* __restrict__ T, const int* __restrict__ tidx,
                                                        float* __restrict__ dS, double* __restrict__ part) {
  __shared__ float2 win[kWS][kWS + 1];   // (I, T) of the window
  __shared__ float2 h01[kWS][kTS + 1];   // row sums (m_I, m_T)
  __shared__ float2 h23[kWS][kTS + 1];   // row sums (m_II, m_TT)
  __shared__ float h4[kWS][kTS + 1];     // row sums m_IT
  __shared__ double red[2][kThreads / 32];
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * kTS, y0 = blockIdx.y * kTS;
  const int64_t HW = (int64_t)p.H * p.W;
  const float* Ip = I + (int64_t)s * HW;
  const float* Tp = T + (int64_t)(tidx ? tidx[s] : s) * HW;
  const float* const src[2] = {Ip, Tp};
  stage_window<2>(p, src, x0, y0, planes_aligned<2>(p, src),
                  [&](int r, int c, const float (&v)[2]) { win[r][c] = make_float2(v[0], v[1]); });
  __syncthreads();
  // horizontal window sums: a thread takes 8 consecutive outputs of one row from
  // 18 staged (I, T) pairs held in registers, the moments of I and T side by
  // side in packed fp32x2 instructions (each lane rounds as the scalar form)
  for (int i = threadIdx.x; i < kWS * (kTS / 8); i += kThreads) {
    const int c0 = (i / kWS) * 8, r = i - (i / kWS) * kWS;  // consecutive lanes: consecutive rows
    float2 u[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = win[r][c0 + k];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      float2 a01 = splat(0.f), a23 = splat(0.f);
      float a4 = 0.f;
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        const float2 w2 = splat(p.w[k]), uv = u[o + k];
        a01 = __ffma2_rn(w2, uv, a01);
        const float2 wuv = __fmul2_rn(w2, uv);
        a23 = __ffma2_rn(wuv, uv, a23);
        a4 = fmaf(wuv.x, uv.y, a4);
      }
      h01[r][c0 + o] = a01;
      h23[r][c0 + o] = a23;
      h4[r][c0 + o] = a4;
    }
  }
  __syncthreads();
  // vertical window sums: a thread takes 4 consecutive outputs of one column,
  // then the SSIM term and its derivatives for each (one division per pixel:
  // 1/C and 1/D come from 1/(C D))
  float ssim_f = 0.f, l1_f = 0.f;  // this thread's four pixels, then a fixed xor tree per warp
  {
    const int i = threadIdx.x;  // kTS * (kTS / 4) == kThreads outputs groups
    const int x = i % kTS, yb = (i / kTS) * 4;
    float2 m01[4], m23[4];
    float m4[4];
    {
      float2 col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = h01[yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float2 acc = splat(0.f);
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = __ffma2_rn(splat(p.w[k]), col[o + k], acc);
        m01[o] = acc;
      }
    }
    {
      float2 col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = h23[yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float2 acc = splat(0.f);
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = __ffma2_rn(splat(p.w[k]), col[o + k], acc);
        m23[o] = acc;
      }
    }
    {
      float col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = h4[yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = fmaf(p.w[k], col[o + k], acc);
        m4[o] = acc;
      }
    }
    const int64_t plane = (int64_t)p.S * HW;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int y = yb + o;
      const int gy = y0 + y, gx = x0 + x;
      if (!in_img(p, gy, gx)) continue;
      const float mI = m01[o].x, mT = m01[o].y;
      const float sII = m23[o].x - mI * mI, sTT = m23[o].y - mT * mT, sIT = m4[o] - mI * mT;
      const float A = fmaf(2.0f * mI, mT, p.c1), Bv = fmaf(2.0f, sIT, p.c2);
      const float Cv = fmaf(mI, mI, fmaf(mT, mT, p.c1)), D = sII + sTT + p.c2;
      const float inv_CD = 1.0f / (Cv * D);
      const float Sv = A * Bv * inv_CD;
      const float dS_dmI = 2.0f * mT * Bv * inv_CD - 2.0f * mI * Sv * (D * inv_CD);  // S 2 m_I / C
      const float dS_dsII = -Sv * (Cv * inv_CD);                                     // -S / D
      const float dS_dsIT = 2.0f * A * inv_CD;
      const int64_t off = (int64_t)s * HW + (int64_t)gy * p.W + gx;
      dS[off] = dS_dmI - 2.0f * mI * dS_dsII - mT * dS_dsIT;  // dS/dm_I (all paths)
      dS[plane + off] = dS_dsII;                              // dS/dm_II
      dS[2 * plane + off] = dS_dsIT;                          // dS/dm_IT
      const float2 it = win[y + kHalo][x + kHalo];
      ssim_f += Sv;
      l1_f += fabsf(it.x - it.y);
    }
  }
  // block sums in a fixed order: fp32 xor trees over the warp's 128 pixels,
  // then the eight warps in double
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ssim_f += __shfl_xor_sync(0xffffffffu, ssim_f, o);
    l1_f += __shfl_xor_sync(0xffffffffu, l1_f, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = (double)ssim_f;
    red[1][threadIdx.x >> 5] = (double)l1_f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[2 * blk] = a;
    part[2 * blk + 1] = b;
  }
}

__global__ void __launch_bounds__(kThreads, 5) k_ssim_grad(SsimArgs p, const float* __restrict__ I,
                                                       const float* __restrict__ T, const int* __restrict__ tidx,
                                                       const float* __restrict__ dS, float* __restrict__ dL_dI) {
  __shared__ float2 sA01[kWS][kWS + 1];  // (dS/dm_I, dS/dm_II) of the window
  __shared__ float sA2[kWS][kWS + 1];    // dS/dm_IT
  __shared__ float2 h01[kWS][kTS + 1];   // their row sums
  __shared__ float h2[kWS][kTS + 1];
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * kTS, y0 = blockIdx.y * kTS;
  const int64_t HW = (int64_t)p.H * p.W;
  const int64_t plane = (int64_t)p.S * HW;
  const float* d0 = dS + (int64_t)s * HW;
  const float* const src[3] = {d0, d0 + plane, d0 + 2 * plane};
  // the thread's four output pixels (column x, rows yb .. yb + 3): their I and T
  // are loaded first, so the epilogue does not wait on them
  const int ox = threadIdx.x % kTS, oyb = (threadIdx.x / kTS) * 4;
  const float* Ip = I + (int64_t)s * HW;
  const float* Tp = T + (int64_t)(tidx ? tidx[s] : s) * HW;
  float iv[4], tv[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int gy = y0 + oyb + o, gx = x0 + ox;
    const bool in = in_img(p, gy, gx);
    const int64_t off = (int64_t)gy * p.W + gx;
    iv[o] = in ? Ip[off] : 0.0f;
    tv[o] = in ? Tp[off] : 0.0f;
  }
  stage_window<3>(p, src, x0, y0, planes_aligned<3>(p, src), [&](int r, int c, const float (&v)[3]) {
    sA01[r][c] = make_float2(v[0], v[1]);
    sA2[r][c] = v[2];
  });
  __syncthreads();
  for (int i = threadIdx.x; i < kWS * (kTS / 8); i += kThreads) {
    const int c0 = (i / kWS) * 8, r = i - (i / kWS) * kWS;  // consecutive lanes: consecutive rows
    float2 u[18];
    float v[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      u[k] = sA01[r][c0 + k];
      v[k] = sA2[r][c0 + k];
    }
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      float2 a = splat(0.f);
      float b = 0.f;
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        a = __ffma2_rn(splat(p.w[k]), u[o + k], a);
        b = fmaf(p.w[k], v[o + k], b);
      }
      h01[r][c0 + o] = a;
      h2[r][c0 + o] = b;
    }
  }
  __syncthreads();
  {
    const int x = ox, yb = oyb;  // kTS * (kTS / 4) == kThreads output groups
    float2 c01[4];
    float c2[4];
    {
      float2 col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = h01[yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float2 acc = splat(0.f);
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = __ffma2_rn(splat(p.w[k]), col[o + k], acc);
        c01[o] = acc;
      }
    }
    {
      float col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = h2[yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = fmaf(p.w[k], col[o + k], acc);
        c2[o] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int gy = y0 + yb + o, gx = x0 + x;
      if (!in_img(p, gy, gx)) continue;
      const int64_t off = (int64_t)gy * p.W + gx;
      const float d = iv[o] - tv[o];
      const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
      const float dssim = fmaf(2.0f * iv[o], c01[o].y, fmaf(tv[o], c2[o], c01[o].x));
      dL_dI[(int64_t)s * HW + off] = p.inv_n * fmaf(-p.lam, dssim, sgn);
    }
  }
}

__global__ void k_ssim_final(const double* __restrict__ part, int64_t nblk, double inv_n, float lam,
                             float* __restrict__ loss) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < nblk; i += 256) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ms = red[0][0] * inv_n, l1 = red[1][0] * inv_n;
    loss[0] = (float)(l1 + (double)lam * (1.0 - ms));
    loss[1] = (float)l1;
    loss[2] = (float)ms;
  }
}

}  // namespace

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_l1_dssim_grad(gp_ctx* ctx, const float* I, const float* T, const int* t_index, int S, int H, int W,
                           float lambda, float* dL_dI, float* loss, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (S < 0 || H <= 0 || W <= 0) return set_err(c, GP_ERR_ARG, "need S >= 0, H > 0, W > 0");
  if (!(lambda >= 0.0f) || !isfinite(lambda)) return set_err(c, GP_ERR_ARG, "lambda must be finite and >= 0");
  if (S == 0) return GP_OK;
  if (!I || !T || !dL_dI) return set_err(c, GP_ERR_ARG, "NULL image pointer");
  if ((int64_t)S * H * W > (int64_t)INT32_MAX) return set_err(c, GP_ERR_ARG, "S*H*W exceeds 2^31");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t npx = (int64_t)S * H * W;
  const dim3 grid((unsigned)((W + kTS - 1) / kTS), (unsigned)((H + kTS - 1) / kTS), (unsigned)S);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  if (grid.z > 65535u) return set_err(c, GP_ERR_ARG, "too many slices for one call (max 65535)");
  BinBufs& b = c->b;
  const size_t ds_bytes = ((size_t)3 * npx * 4 + 255) & ~(size_t)255;
  const size_t part_bytes = ((size_t)nblk * 16 + 255) & ~(size_t)255;
  gp_status rs = ws_reserve(c, b.loss_tmp, ds_bytes + part_bytes + (size_t)S * 4 + 64);
  if (rs != GP_OK) return rs;
  char* base = (char*)b.loss_tmp.ptr;
  float* dS = (float*)base;
  double* part = (double*)(base + ds_bytes);
  int* tid = nullptr;
  if (t_index) {
    for (int s = 0; s < S; ++s)
      if (t_index[s] < 0) return set_err(c, GP_ERR_ARG, "negative target slice index");
    tid = (int*)(base + ds_bytes + part_bytes);
    uint32_t* d1[1] = {(uint32_t*)tid};
    const void* s1[1] = {t_index};
    if (put_words(st, 1, d1, s1, &S) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "upload t_index");
  }
  SsimArgs p;
  double w[11], sum = 0.0;
  for (int k = 0; k < 11; ++k) {
    const double x = (double)(k - 5);
    w[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
    sum += w[k];
  }
  for (int k = 0; k < 11; ++k) p.w[k] = (float)(w[k] / sum);
  p.S = S; p.H = H; p.W = W;
  p.c1 = 1e-4f; p.c2 = 9e-4f;
  p.inv_n = (float)(1.0 / (double)npx);
  p.lam = lambda;
  PhaseTimer timer(c, GP_PHASE_LOSS, st);
  k_ssim_stats<<<grid, kThreads, 0, st>>>(p, I, T, tid, dS, part);
  k_ssim_grad<<<grid, kThreads, 0, st>>>(p, I, T, tid, dS, dL_dI);
  note_launch(2);
  if (loss) {
    k_ssim_final<<<1, 256, 0, st>>>(part, nblk, 1.0 / (double)npx, lambda, loss);
    note_launch();
  }
  return cuda_err(c, cudaGetLastError(), "l1 + d-ssim");
}

}  // extern "C"
