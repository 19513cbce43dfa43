// raster.cu -- block-culled tile rasterisers of the slice renderer (the default
// K-fwd and K-bwd for 16 x 16 tiles), sm_103a.
//
// A CTA owns one (slice, 16x16 tile) and its binned Gaussian list; its four
// warps own the four 8x8 blocks of the tile.  Per round the CTA stages a chunk
// of Gaussians in shared memory (16-byte loads of the 64-byte records, mu_2d
// and a~ of this slice computed once per Gaussian).  Each warp then tests 32
// staged Gaussians at a time against its block -- lane l tests Gaussian l with
//     || c - mu_2d ||_C  >  k + max_{p in block} || p - c ||_C
// (c the block centre, ||x||_C^2 = x^T Sigma_2d^-1 x, k^2 = 2 ln(1/eps)), which
// by the triangle inequality proves every pixel of the block lies outside the
// culling ellipse -- and compacts the hits with a ballot.  The warp's four
// 8-lane groups then take four hits at a time; lane r of a group evaluates row r
// of the block (8 pixels), so the per-Gaussian terms (row offset, shared part
// of the quadratic form) are paid once per 8 pixels and the backward's
// per-Gaussian reductions are 8-lane trees.
//
// Forward: each lane keeps 8 partial sums per group; the four groups are added
// in a fixed shuffle tree at the end, so results are bitwise reproducible.
// Backward: six pixel moments per (Gaussian, block) -- sum G E, sum G E dx,
// sum G E dy, sum G E dx^2, sum G E dx dy, sum G E dy^2 with E the Gaussian's
// exponential and G = dL/dI -- reduced over the group's 8 rows, stored per warp,
// summed over the 4 warps in a fixed order, then folded into the 10
// accumulators of the Gaussian (atomics) or written as a per-pair partial
// (deterministic mode).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_common.cuh"
#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

constexpr int BT = 16;          // tile side
constexpr int BNT = 128;        // threads per CTA: 4 warps, one 8x8 block each
constexpr int FCH = 128;        // Gaussians staged per round, forward
constexpr int BCH = 64;         // Gaussians staged per round, backward
constexpr float kHalfBlock = 3.5f;  // pixel centres of an 8-wide block lie within +-3.5 of its centre

// Staging of one Gaussian for one (slice, tile):
//   s0 = (mu_2d,x - x0, mu_2d,y - y0, a~, thr)   thr: block-cull threshold (base-2 exponent units)
//   s1 = (c0, c1, c2, C00)                        e = c0 dx^2 + c1 dx dy + c2 dy^2 = -log2(e)/2 d^T C d
//   s2 = (delta, opacity_r, C01, C11)             backward only
template <int EXPM>
__device__ __forceinline__ void stage_blk(const SliceRec* __restrict__ rec, uint32_t g, float zsv, float x0,
                                          float y0, float sqrt_k2, float4& s0, float4& s1, float4& s2) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2);
  const float d = r0.z - zsv;
  const float w = exp2_sel<EXPM>(fmaxf(-0.5f * kLog2e * d * d * r0.w, kExpFloor));
  const float mxr = (r0.x - x0) - r1.x * d;
  const float myr = (r0.y - y0) - r1.y * d;
  const float C00 = r2.x, C01 = r2.y, C11 = r2.z;
  const float R2 = kHalfBlock * kHalfBlock * (C00 + C11) + 2.0f * kHalfBlock * kHalfBlock * fabsf(C01);
  const float kr = sqrt_k2 + sqrtf(R2);
  s0 = make_float4(mxr, myr, r1.z * w, -0.5f * kLog2e * kr * kr);
  s1 = make_float4(-0.5f * kLog2e * C00, -kLog2e * C01, -0.5f * kLog2e * C11, C00);
  s2 = make_float4(d, w, C01, C11);
}

// Ballot of the Gaussians jb..jb+31 that may touch this warp's block; their
// chunk indices are compacted into list[0..n).  Returns n.
__device__ __forceinline__ int block_hits(const float4* __restrict__ s0, const float4* __restrict__ s1, int jb,
                                          int cnt, float cx, float cy, int lane, int* list) {
  const int j = jb + lane;
  bool hit = false;
  if (j < cnt) {
    const float4 g0 = s0[j], g1 = s1[j];
    const float dx = cx - g0.x, dy = cy - g0.y;
    const float e = fmaf(dx, fmaf(g1.x, dx, g1.y * dy), g1.z * dy * dy);
    hit = e >= g0.w;
  }
  const unsigned m = __ballot_sync(0xffffffffu, hit);
  if (hit) list[__popc(m & ((1u << lane) - 1u))] = j;
  __syncwarp();
  return __popc(m);
}

template <int EXPM>
__global__ void __launch_bounds__(BNT) k_raster_fwd_blk(SliceArgs a, const SliceRec* __restrict__ rec,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ emit_gid,
                                                        const uint2* __restrict__ ranges, float* __restrict__ out) {
  __shared__ float4 s0[FCH], s1[FCH];
  __shared__ int hitlist[BNT / 32][32];
  const int T = a.TX * a.TY;
  const int tile_id = blockIdx.x;
  const int s = tile_id / T, t = tile_id - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const uint2 rg = ranges[tile_id];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> 3, row = lane & 7;
  const float bx = (float)((warp & 1) * 8), by = (float)((warp >> 1) * 8);
  const float cx = bx + 4.0f, cy = by + 4.0f;
  const float pyr = by + (float)row + 0.5f;
  const float x0 = (float)(tx * BT), y0 = (float)(ty * BT);
  const float zsv = a.zorig[s];
  const float sqrt_k2 = sqrtf(a.k2);
  int* list = hitlist[warp];
  float acc[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) acc[p] = 0.0f;
  for (uint32_t base = rg.x; base < rg.y; base += FCH) {
    const int cnt = (int)min((uint32_t)FCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += BNT) {
      float4 a0, a1, a2;
      stage_blk<EXPM>(rec, emit_gid[vals[base + j]], zsv, x0, y0, sqrt_k2, a0, a1, a2);
      s0[j] = a0;
      s1[j] = a1;
    }
    __syncthreads();
    for (int jb = 0; jb < cnt; jb += 32) {
      const int nh = block_hits(s0, s1, jb, cnt, cx, cy, lane, list);
      for (int h = grp; h < nh; h += 4) {
        const int jj = list[h];
        const float4 g0 = s0[jj], g1 = s1[jj];
        const float dy = pyr - g0.y;
        const float u = g1.y * dy;
        const float wy = g1.z * dy * dy;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const float dx = (bx + (float)p + 0.5f) - g0.x;
          float e = fmaf(dx, fmaf(g1.x, dx, u), wy);
          e = fmaxf(e, kExpFloor);
          acc[p] = fmaf(g0.z, exp2_sel<EXPM>(e), acc[p]);
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // the four groups' partial sums of the same pixels, in a fixed tree
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], 8);
    acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], 16);
  }
  if (grp == 0) {
    const int py = ty * BT + (int)by + row;
    const int px0 = tx * BT + (int)bx;
    if (py < a.H) {
      float* o = out + ((int64_t)s * a.H + py) * a.W + px0;
      if (px0 + 8 <= a.W && ((((uintptr_t)o) & 15u) == 0)) {
        reinterpret_cast<float4*>(o)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        reinterpret_cast<float4*>(o)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      } else {
#pragma unroll
        for (int p = 0; p < 8; ++p)
          if (px0 + p < a.W) o[p] = acc[p];
      }
    }
  }
}

constexpr int ACC10 = 10;

template <int EXPM, bool DET>
__global__ void __launch_bounds__(BNT) k_raster_bwd_blk(SliceArgs a, const SliceRec* __restrict__ rec,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ emit_gid,
                                                        const uint2* __restrict__ ranges,
                                                        const float* __restrict__ dL_dI, float* __restrict__ accum,
                                                        float4* __restrict__ partial) {
  constexpr int NW = BNT / 32;
  __shared__ float4 s0[BCH], s1[BCH], s2[BCH];
  __shared__ uint32_t sg[BCH];
  __shared__ float sp[NW][6][BCH];
  __shared__ int hitlist[NW][32];
  const int T = a.TX * a.TY;
  const int tile_id = blockIdx.x;
  const uint2 rg = ranges[tile_id];
  if (rg.y <= rg.x) return;
  const int s = tile_id / T, t = tile_id - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> 3, row = lane & 7;
  const unsigned gmask = 0xffu << (grp * 8);
  const float bx = (float)((warp & 1) * 8), by = (float)((warp >> 1) * 8);
  const float cx = bx + 4.0f, cy = by + 4.0f;
  const float pyr = by + (float)row + 0.5f;
  const float x0 = (float)(tx * BT), y0 = (float)(ty * BT);
  const float zsv = a.zorig[s];
  const float sqrt_k2 = sqrtf(a.k2);
  int* list = hitlist[warp];
  float G[8];
  {
    const int py = ty * BT + (int)by + row;
    const int px0 = tx * BT + (int)bx;
#pragma unroll
    for (int p = 0; p < 8; ++p)
      G[p] = (py < a.H && px0 + p < a.W) ? dL_dI[((int64_t)s * a.H + py) * a.W + px0 + p] : 0.0f;
  }
  for (uint32_t base = rg.x; base < rg.y; base += BCH) {
    const int cnt = (int)min((uint32_t)BCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += BNT) {
      const uint32_t g = emit_gid[vals[base + j]];
      float4 a0, a1, a2;
      stage_blk<EXPM>(rec, g, zsv, x0, y0, sqrt_k2, a0, a1, a2);
      s0[j] = a0;
      s1[j] = a1;
      s2[j] = a2;
      sg[j] = g;
    }
    for (int i = threadIdx.x; i < NW * 6 * BCH; i += BNT) (&sp[0][0][0])[i] = 0.0f;
    __syncthreads();
    for (int jb = 0; jb < cnt; jb += 32) {
      const int nh = block_hits(s0, s1, jb, cnt, cx, cy, lane, list);
      for (int h = grp; h < nh; h += 4) {
        const int jj = list[h];
        const float4 g0 = s0[jj], g1 = s1[jj];
        const float dy = pyr - g0.y;
        const float u = g1.y * dy;
        const float wy = g1.z * dy * dy;
        float m0 = 0.f, mx = 0.f, mxx = 0.f;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const float dx = (bx + (float)p + 0.5f) - g0.x;
          float e = fmaf(dx, fmaf(g1.x, dx, u), wy);
          e = fmaxf(e, kExpFloor);
          const float gE = G[p] * exp2_sel<EXPM>(e);
          m0 += gE;
          const float tdx = gE * dx;
          mx += tdx;
          mxx = fmaf(tdx, dx, mxx);
        }
        float v[6] = {m0, mx, m0 * dy, mxx, mx * dy, m0 * dy * dy};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          v[k] += __shfl_xor_sync(gmask, v[k], 1);
          v[k] += __shfl_xor_sync(gmask, v[k], 2);
          v[k] += __shfl_xor_sync(gmask, v[k], 4);
        }
        if (row == 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) sp[warp][k][jj] = v[k];
        }
      }
      __syncwarp();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += BNT) {
      float m[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) acc += sp[w][k][j];
        m[k] = acc;
      }
      const float4 g0 = s0[j], g1 = s1[j], g2 = s2[j];
      const float at = g0.z;
      const float C00 = g1.w, C01 = g2.z, C11 = g2.w;
      // dE/dmu_2d = E C d; dE/dC00 = -E dx^2/2, dE/dC01 = -E dx dy, dE/dC11 = -E dy^2/2
      const float g_at = m[0];
      const float gmx = at * (C00 * m[1] + C01 * m[2]);
      const float gmy = at * (C01 * m[1] + C11 * m[2]);
      const float gc00 = -0.5f * at * m[3];
      const float gc01 = -at * m[4];
      const float gc11 = -0.5f * at * m[5];
      const float d = g2.x, w = g2.y;
      if constexpr (DET) {
        const uint32_t e = vals[base + j];
        partial[2 * (size_t)e] = make_float4(g_at, gmx, gmy, gc00);
        partial[2 * (size_t)e + 1] = make_float4(gc01, gc11, d, w);
      } else {
        float* A = accum + (size_t)sg[j] * ACC10;
        const float gw = g_at * w;
        atomicAdd(A + 0, gmx);
        atomicAdd(A + 1, gmy);
        atomicAdd(A + 2, d * gmx);
        atomicAdd(A + 3, d * gmy);
        atomicAdd(A + 4, gw);
        atomicAdd(A + 5, gw * d);
        atomicAdd(A + 6, gw * d * d);
        atomicAdd(A + 7, gc00);
        atomicAdd(A + 8, gc01);
        atomicAdd(A + 9, gc11);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_raster_fwd_blocked(const SliceArgs& a, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                                      const uint32_t* emit_gid, const uint2* ranges, float* out, cudaStream_t st) {
  const int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  if (tiles == 0) return cudaSuccess;
  if (a.tile != BT) return cudaErrorInvalidValue;
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd_blk<GP_EXP_HW><<<(unsigned)tiles, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, out);
  else
    k_raster_fwd_blk<GP_EXP_POLY><<<(unsigned)tiles, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd_blocked(const SliceArgs& a, int exp_mode, bool det, const SliceRec* rec,
                                      const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                      const float* dL_dI, float* accum, float4* partial, cudaStream_t st) {
  const int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  if (tiles == 0) return cudaSuccess;
  if (a.tile != BT) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)tiles;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd_blk<GP_EXP_HW, true><<<g, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
    else k_raster_bwd_blk<GP_EXP_HW, false><<<g, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
  } else {
    if (det) k_raster_bwd_blk<GP_EXP_POLY, true><<<g, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
    else k_raster_bwd_blk<GP_EXP_POLY, false><<<g, BNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace gp
