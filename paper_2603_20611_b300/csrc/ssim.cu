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
// About 44 bytes of HBM traffic per pixel in all: a memory-bound loss, ~1 % of
// a fit step.
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

struct SsimArgs {
  float w[11];  // 1-D window, normalised to sum 1
  int S, H, W;
  float c1, c2, inv_n, lam;
};

__device__ __forceinline__ bool in_img(const SsimArgs& p, int y, int x) {
  return y >= 0 && y < p.H && x >= 0 && x < p.W;
}

__global__ void __launch_bounds__(kThreads) k_ssim_stats(SsimArgs p, const float* __restrict__ I,
                                                        const float* __restrict__ T, const int* __restrict__ tidx,
                                                        float* __restrict__ dS, double* __restrict__ part) {
  __shared__ float sI[kWS][kWS + 1], sT[kWS][kWS + 1];
  __shared__ float hs[5][kWS][kTS + 1];
  __shared__ double red[2][kThreads / 32];
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * kTS, y0 = blockIdx.y * kTS;
  const int64_t HW = (int64_t)p.H * p.W;
  const float* Ip = I + (int64_t)s * HW;
  const float* Tp = T + (int64_t)(tidx ? tidx[s] : s) * HW;
  for (int i = threadIdx.x; i < kWS * kWS; i += kThreads) {
    const int r = i / kWS, c = i - r * kWS;
    const int y = y0 - kHalo + r, x = x0 - kHalo + c;
    const bool in = in_img(p, y, x);
    sI[r][c] = in ? Ip[(int64_t)y * p.W + x] : 0.0f;
    sT[r][c] = in ? Tp[(int64_t)y * p.W + x] : 0.0f;
  }
  __syncthreads();
  // horizontal window sums: a thread takes 8 consecutive outputs of one row from
  // 18 staged values of each image (a sliding window held in registers)
  for (int i = threadIdx.x; i < kWS * (kTS / 8); i += kThreads) {
    const int r = i / (kTS / 8), c0 = (i - r * (kTS / 8)) * 8;
    float u[18], v[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      u[k] = sI[r][c0 + k];
      v[k] = sT[r][c0 + k];
    }
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        const float wk = p.w[k], uu = u[o + k], vv = v[o + k];
        a0 = fmaf(wk, uu, a0);
        a1 = fmaf(wk, vv, a1);
        a2 = fmaf(wk * uu, uu, a2);
        a3 = fmaf(wk * vv, vv, a3);
        a4 = fmaf(wk * uu, vv, a4);
      }
      hs[0][r][c0 + o] = a0; hs[1][r][c0 + o] = a1; hs[2][r][c0 + o] = a2; hs[3][r][c0 + o] = a3;
      hs[4][r][c0 + o] = a4;
    }
  }
  __syncthreads();
  double ssim_acc = 0.0, l1_acc = 0.0;
  // vertical window sums: a thread takes 4 consecutive outputs of one column
  for (int i = threadIdx.x; i < kTS * (kTS / 4); i += kThreads) {
    const int x = i % kTS, yb = (i / kTS) * 4;
    float mm[4][5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      float col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = hs[q][yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = fmaf(p.w[k], col[o + k], acc);
        mm[o][q] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
    const int y = yb + o;
    const int gy = y0 + y, gx = x0 + x;
    if (!in_img(p, gy, gx)) continue;
    const float* m = mm[o];
    const float mI = m[0], mT = m[1];
    const float sII = m[2] - mI * mI, sTT = m[3] - mT * mT, sIT = m[4] - mI * mT;
    const float A = fmaf(2.0f * mI, mT, p.c1), Bv = fmaf(2.0f, sIT, p.c2);
    const float Cv = fmaf(mI, mI, fmaf(mT, mT, p.c1)), D = sII + sTT + p.c2;
    const float inv_CD = 1.0f / (Cv * D);
    const float Sv = A * Bv * inv_CD;
    const float dS_dmI = 2.0f * mT * Bv * inv_CD - Sv * 2.0f * mI / Cv;
    const float dS_dsII = -Sv / D;
    const float dS_dsIT = 2.0f * A * inv_CD;
    const int64_t off = (int64_t)s * HW + (int64_t)gy * p.W + gx;
    const int64_t plane = (int64_t)p.S * HW;
    dS[off] = dS_dmI - 2.0f * mI * dS_dsII - mT * dS_dsIT;  // dS/dm_I (all paths)
    dS[plane + off] = dS_dsII;                              // dS/dm_II
    dS[2 * plane + off] = dS_dsIT;                          // dS/dm_IT
    ssim_acc += (double)Sv;
    l1_acc += (double)fabsf(sI[y + kHalo][x + kHalo] - sT[y + kHalo][x + kHalo]);
    }
  }
  // block sums in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ssim_acc += __shfl_xor_sync(0xffffffffu, ssim_acc, o);
    l1_acc += __shfl_xor_sync(0xffffffffu, l1_acc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ssim_acc;
    red[1][threadIdx.x >> 5] = l1_acc;
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

__global__ void __launch_bounds__(kThreads) k_ssim_grad(SsimArgs p, const float* __restrict__ I,
                                                       const float* __restrict__ T, const int* __restrict__ tidx,
                                                       const float* __restrict__ dS, float* __restrict__ dL_dI) {
  __shared__ float sA[3][kWS][kWS + 1];
  __shared__ float hs[3][kWS][kTS + 1];
  const int s = blockIdx.z;
  const int x0 = blockIdx.x * kTS, y0 = blockIdx.y * kTS;
  const int64_t HW = (int64_t)p.H * p.W;
  const int64_t plane = (int64_t)p.S * HW;
  for (int i = threadIdx.x; i < kWS * kWS; i += kThreads) {
    const int r = i / kWS, c = i - r * kWS;
    const int y = y0 - kHalo + r, x = x0 - kHalo + c;
    const bool in = in_img(p, y, x);
    const int64_t o = (int64_t)s * HW + (int64_t)y * p.W + x;
#pragma unroll
    for (int q = 0; q < 3; ++q) sA[q][r][c] = in ? dS[q * plane + o] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * kWS * (kTS / 8); i += kThreads) {
    const int q = i / (kWS * (kTS / 8));
    const int rr = i - q * (kWS * (kTS / 8));
    const int r = rr / (kTS / 8), c0 = (rr - r * (kTS / 8)) * 8;
    float u[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = sA[q][r][c0 + k];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 11; ++k) acc = fmaf(p.w[k], u[o + k], acc);
      hs[q][r][c0 + o] = acc;
    }
  }
  __syncthreads();
  const float* Ip = I + (int64_t)s * HW;
  const float* Tp = T + (int64_t)(tidx ? tidx[s] : s) * HW;
  for (int i = threadIdx.x; i < kTS * (kTS / 4); i += kThreads) {
    const int x = i % kTS, yb = (i / kTS) * 4;
    float cc[4][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float col[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) col[k] = hs[q][yb + k][x];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) acc = fmaf(p.w[k], col[o + k], acc);
        cc[o][q] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
    const int y = yb + o;
    const int gy = y0 + y, gx = x0 + x;
    if (!in_img(p, gy, gx)) continue;
    const float* c = cc[o];
    const int64_t off = (int64_t)gy * p.W + gx;
    const float iv = Ip[off], tv = Tp[off];
    const float d = iv - tv;
    const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
    const float dssim = fmaf(2.0f * iv, c[1], fmaf(tv, c[2], c[0]));
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
