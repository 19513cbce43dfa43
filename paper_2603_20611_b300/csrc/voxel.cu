// voxel.cu -- sm_103a kernels of the differentiable voxelizer (GaussianPile,
// arXiv 2603.20611, Sec. 4.3 "Differentiable Voxelization", Eq. 12):
//     V(x) = sum_i alpha_i exp(-1/2 (x - mu_i)^T Sigma_i^-1 (x - mu_i))
// on a voxel grid partitioned into 8^3 tiles.
//
// Pipeline (the sort and scan are shared with the slice renderer):
//   K-vpre   per Gaussian: record (mu, alpha, K = Sigma^-1, bounding box of the
//            ellipsoid (x-mu)^T K (x-mu) <= 2 ln(1/eps)) + number of tiles
//   K-vemit  tile keys with emission indices
//   K-vfwd   one 64-thread CTA per tile; each thread owns one (x, y) column of
//            eight voxels, so the x/y part of the quadratic form is computed once
//            per Gaussian and each voxel costs two FMAs plus the exponential
//   K-vbwd   ten moments per (Gaussian, tile) (sum G E, sum G E d_i,
//            sum G E d_i d_j), warp-reduced, summed over the two warps in a
//            fixed order, then atomically added per Gaussian (or stored per pair
//            for the deterministic ordered reduction)
//   K-vbwd-pre  moments -> dL/d(mu, scale, quat, alpha)
#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_common.cuh"
#include "gp_internal.h"
#include "voxel.cuh"

namespace gp {

constexpr int VPRE_THREADS = 256;
constexpr int VNT = 64;      // threads per voxel tile
constexpr int VCH = 128;     // Gaussians staged per round
constexpr int VACC = 10;     // moments per Gaussian

// inverse of a symmetric 3x3 (xx, xy, xz, yy, yz, zz) by cofactors
__device__ __forceinline__ float sym_inv3(const float S[6], float K[6]) {
  float c00 = S[3] * S[5] - S[4] * S[4];
  float c01 = S[2] * S[4] - S[1] * S[5];
  float c02 = S[1] * S[4] - S[2] * S[3];
  float det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  float id = 1.0f / det;
  K[0] = c00 * id;
  K[1] = c01 * id;
  K[2] = c02 * id;
  K[3] = (S[0] * S[5] - S[2] * S[2]) * id;
  K[4] = (S[1] * S[2] - S[0] * S[4]) * id;
  K[5] = (S[0] * S[3] - S[1] * S[1]) * id;
  return det;
}

struct TileBox {
  int x0, x1, y0, y1, z0, z1;
};

__device__ __forceinline__ int vclamp(float t, int nt) {
  t = fminf(fmaxf(t, -1.0f), (float)nt);
  return (int)floorf(t);
}

__device__ __forceinline__ TileBox vox_tiles(const VoxArgs& a, const VoxRec& r) {
  TileBox b;
  const float inv = 1.0f / (float)VOX_TILE;
  b.x0 = max(0, vclamp(__fmul_rn(__fsub_rn(__fsub_rn(r.r0.x, r.r2.z), 0.5f), inv), a.TX));
  b.x1 = min(a.TX - 1, vclamp(__fmul_rn(__fsub_rn(__fadd_rn(r.r0.x, r.r2.z), 0.5f), inv), a.TX));
  b.y0 = max(0, vclamp(__fmul_rn(__fsub_rn(__fsub_rn(r.r0.y, r.r2.w), 0.5f), inv), a.TY));
  b.y1 = min(a.TY - 1, vclamp(__fmul_rn(__fsub_rn(__fadd_rn(r.r0.y, r.r2.w), 0.5f), inv), a.TY));
  b.z0 = max(0, vclamp(__fmul_rn(__fsub_rn(__fsub_rn(r.r0.z, r.r3.x), 0.5f), inv), a.TZ));
  b.z1 = min(a.TZ - 1, vclamp(__fmul_rn(__fsub_rn(__fadd_rn(r.r0.z, r.r3.x), 0.5f), inv), a.TZ));
  return b;
}

__global__ void __launch_bounds__(VPRE_THREADS) k_vox_pre(VoxArgs a, VoxRec* __restrict__ rec,
                                                          unsigned long long* __restrict__ counts) {
  int i = blockIdx.x * VPRE_THREADS + threadIdx.x;
  if (i >= a.n) return;
  float4 q = reinterpret_cast<const float4*>(a.quat)[i];
  float R[3][3], qn[4], qnorm;
  quat_rot(q, R, qn, qnorm);
  float d3[3] = {a.mod * a.scale[3 * i], a.mod * a.scale[3 * i + 1], a.mod * a.scale[3 * i + 2]};
  float M[3][3], Sw[6], K[6];
  covariance(R, d3, M, Sw);
  float det = sym_inv3(Sw, K);
  float mx = a.mu[3 * i], my = a.mu[3 * i + 1], mz = a.mu[3 * i + 2];
  bool valid = det > 1e-30f && isfinite(det) && qnorm > 0.0f && isfinite(mx) && isfinite(my) &&
               isfinite(mz) && isfinite(a.alpha[i]);
  VoxRec r;
  r.r0 = make_float4(mx, my, mz, a.alpha[i]);
  r.r1 = make_float4(K[0], K[1], K[2], K[3]);
  r.r2 = make_float4(K[4], K[5], sqrtf(a.k2 * Sw[0]), sqrtf(a.k2 * Sw[3]));
  r.r3 = make_float4(sqrtf(a.k2 * Sw[5]), valid ? 1.0f : 0.0f, 0.0f, 0.0f);
  rec[i] = r;
  unsigned long long cnt = 0;
  if (valid) {
    TileBox b = vox_tiles(a, r);
    if (b.x1 >= b.x0 && b.y1 >= b.y0 && b.z1 >= b.z0)
      cnt = (unsigned long long)(b.x1 - b.x0 + 1) * (b.y1 - b.y0 + 1) * (b.z1 - b.z0 + 1);
  }
  counts[i] = cnt;
}

void launch_vox_pre(const VoxArgs& a, VoxRec* rec, unsigned long long* counts, cudaStream_t st) {
  if (a.n <= 0) return;
  k_vox_pre<<<ceil_div(a.n, VPRE_THREADS), VPRE_THREADS, 0, st>>>(a, rec, counts);
  note_launch();
}

__global__ void __launch_bounds__(VPRE_THREADS) k_vox_emit(VoxArgs a, const VoxRec* __restrict__ rec,
                                                           const unsigned long long* __restrict__ offsets,
                                                           const unsigned long long* __restrict__ counts,
                                                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                           uint32_t* __restrict__ emit_gid) {
  int i = blockIdx.x * VPRE_THREADS + threadIdx.x;
  if (i >= a.n) return;
  VoxRec r = rec[i];
  if (r.r3.y == 0.0f) return;
  TileBox b = vox_tiles(a, r);
  uint32_t e = (uint32_t)offsets[i];
  const uint32_t e_end = (uint32_t)(offsets[i] + counts[i]);  // never write past this Gaussian's slots
  for (int tz = b.z0; tz <= b.z1; ++tz)
    for (int ty = b.y0; ty <= b.y1; ++ty)
      for (int tx = b.x0; tx <= b.x1; ++tx) {
        if (e < e_end) {
          keys[e] = (uint32_t)((tz * a.TY + ty) * a.TX + tx);
          emit_gid[e] = (uint32_t)i;
        }
        ++e;
      }
}

void launch_vox_emit(const VoxArgs& a, const VoxRec* rec, const unsigned long long* offsets,
                     const unsigned long long* counts, uint32_t* keys, uint32_t* vals, uint32_t* emit_gid,
                     cudaStream_t st) {
  if (a.n <= 0) return;
  k_vox_emit<<<ceil_div(a.n, VPRE_THREADS), VPRE_THREADS, 0, st>>>(a, rec, offsets, counts, keys, vals, emit_gid);
  note_launch();
}

// Staging: mean relative to the tile origin (exact), alpha, and the quadratic
// form pre-scaled to base 2 with doubled off-diagonals:
//   e = q0 dx^2 + q1 dy^2 + q2 dz^2 + q3 dx dy + q4 dx dz + q5 dy dz.
__device__ __forceinline__ void vstage(const VoxRec* __restrict__ rec, uint32_t g, float ox, float oy, float oz,
                                       float4& s0, float4& s1, float2& s2) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2);
  const float h = -0.5f * kLog2e;
  s0 = make_float4(r0.x - ox, r0.y - oy, r0.z - oz, r0.w);
  s1 = make_float4(h * r1.x, h * r1.w, h * r2.y, 2.0f * h * r1.y);  // q0 (xx), q1 (yy), q2 (zz), q3 (xy)
  s2 = make_float2(2.0f * h * r1.z, 2.0f * h * r2.x);                // q4 (xz), q5 (yz)
}

__global__ void __launch_bounds__(VNT) k_vox_fwd(VoxArgs a, const VoxRec* __restrict__ rec,
                                                 const uint32_t* __restrict__ vals,
                                                 const uint32_t* __restrict__ emit_gid,
                                                 const uint2* __restrict__ ranges, float* __restrict__ vol) {
  __shared__ float4 s0[VCH], s1[VCH];
  __shared__ float2 s2[VCH];
  const int tile = blockIdx.x;
  const int tx = tile % a.TX, ty = (tile / a.TX) % a.TY, tz = tile / (a.TX * a.TY);
  const uint2 rg = ranges[tile];
  const int lx = threadIdx.x & 7, ly = threadIdx.x >> 3;
  const float ox = (float)(tx * VOX_TILE), oy = (float)(ty * VOX_TILE), oz = (float)(tz * VOX_TILE);
  const float px = (float)lx + 0.5f, py = (float)ly + 0.5f;
  float acc[VOX_TILE];
#pragma unroll
  for (int k = 0; k < VOX_TILE; ++k) acc[k] = 0.f;
  for (uint32_t base = rg.x; base < rg.y; base += VCH) {
    const int cnt = (int)min((uint32_t)VCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += VNT) {
      uint32_t g = emit_gid[vals[base + j]];
      float4 a0, a1;
      float2 a2;
      vstage(rec, g, ox, oy, oz, a0, a1, a2);
      s0[j] = a0;
      s1[j] = a1;
      s2[j] = a2;
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float4 g0 = s0[j], g1 = s1[j];
      const float2 g2 = s2[j];
      const float dx = px - g0.x, dy = py - g0.y;
      const float bxy = fmaf(dx, fmaf(g1.x, dx, g1.w * dy), g1.y * dy * dy);
      const float lin = fmaf(g2.x, dx, g2.y * dy);
#pragma unroll
      for (int k = 0; k < VOX_TILE; ++k) {
        const float dz = ((float)k + 0.5f) - g0.z;
        float e = fmaf(dz, fmaf(g1.z, dz, lin), bxy);
        e = fmaxf(e, kExpFloor);
        acc[k] = fmaf(g0.w, exp2_poly(e), acc[k]);
      }
    }
    __syncthreads();
  }
  const int x = tx * VOX_TILE + lx, y = ty * VOX_TILE + ly;
  if (x < a.X && y < a.Y) {
#pragma unroll
    for (int k = 0; k < VOX_TILE; ++k) {
      const int z = tz * VOX_TILE + k;
      if (z < a.Z) vol[((int64_t)z * a.Y + y) * a.X + x] = acc[k];
    }
  }
}

cudaError_t launch_vox_fwd(const VoxArgs& a, const VoxRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                           const uint2* ranges, float* vol, cudaStream_t st) {
  int64_t tiles = (int64_t)a.TX * a.TY * a.TZ;
  if (tiles == 0) return cudaSuccess;
  k_vox_fwd<<<(unsigned)tiles, VNT, 0, st>>>(a, rec, vals, emit_gid, ranges, vol);
  note_launch();
  return cudaGetLastError();
}

__device__ __forceinline__ float vwarp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Moment layout: 0 sum G E, 1..3 sum G E (dx, dy, dz),
//                4..9 sum G E (dx dx, dy dy, dz dz, dx dy, dx dz, dy dz).
template <bool DET>
__global__ void __launch_bounds__(VNT) k_vox_bwd(VoxArgs a, const VoxRec* __restrict__ rec,
                                                 const uint32_t* __restrict__ vals,
                                                 const uint32_t* __restrict__ emit_gid,
                                                 const uint2* __restrict__ ranges, const float* __restrict__ dL_dV,
                                                 float* __restrict__ accum, float4* __restrict__ partial) {
  constexpr int NW = VNT / 32;
  __shared__ float4 s0[VCH], s1[VCH];
  __shared__ float2 s2[VCH];
  __shared__ uint32_t sg[VCH];
  __shared__ float sp[NW][VACC][VCH];
  const int tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  if (rg.y <= rg.x) return;
  const int tx = tile % a.TX, ty = (tile / a.TX) % a.TY, tz = tile / (a.TX * a.TY);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & 7, ly = threadIdx.x >> 3;
  const float ox = (float)(tx * VOX_TILE), oy = (float)(ty * VOX_TILE), oz = (float)(tz * VOX_TILE);
  const float px = (float)lx + 0.5f, py = (float)ly + 0.5f;
  const int x = tx * VOX_TILE + lx, y = ty * VOX_TILE + ly;
  float G[VOX_TILE];
#pragma unroll
  for (int k = 0; k < VOX_TILE; ++k) {
    const int z = tz * VOX_TILE + k;
    G[k] = (x < a.X && y < a.Y && z < a.Z) ? dL_dV[((int64_t)z * a.Y + y) * a.X + x] : 0.f;
  }
  for (uint32_t base = rg.x; base < rg.y; base += VCH) {
    const int cnt = (int)min((uint32_t)VCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += VNT) {
      uint32_t g = emit_gid[vals[base + j]];
      float4 a0, a1;
      float2 a2;
      vstage(rec, g, ox, oy, oz, a0, a1, a2);
      s0[j] = a0;
      s1[j] = a1;
      s2[j] = a2;
      sg[j] = g;
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float4 g0 = s0[j], g1 = s1[j];
      const float2 g2 = s2[j];
      const float dx = px - g0.x, dy = py - g0.y;
      const float bxy = fmaf(dx, fmaf(g1.x, dx, g1.w * dy), g1.y * dy * dy);
      const float lin = fmaf(g2.x, dx, g2.y * dy);
      float c0 = 0.f, cz = 0.f, czz = 0.f;
#pragma unroll
      for (int k = 0; k < VOX_TILE; ++k) {
        const float dz = ((float)k + 0.5f) - g0.z;
        float e = fmaf(dz, fmaf(g1.z, dz, lin), bxy);
        e = fmaxf(e, kExpFloor);
        const float gE = G[k] * exp2_poly(e);
        c0 += gE;
        const float t = gE * dz;
        cz += t;
        czz = fmaf(t, dz, czz);
      }
      float m[VACC] = {c0, c0 * dx, c0 * dy, cz, c0 * dx * dx, c0 * dy * dy, czz, c0 * dx * dy, cz * dx, cz * dy};
#pragma unroll
      for (int k = 0; k < VACC; ++k) m[k] = vwarp_sum(m[k]);
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < VACC; ++k) sp[warp][k][j] = m[k];
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += VNT) {
      float m[VACC];
#pragma unroll
      for (int k = 0; k < VACC; ++k) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += sp[w][k][j];
        m[k] = s;
      }
      if constexpr (DET) {
        const size_t e = vals[base + j];
        partial[3 * e] = make_float4(m[0], m[1], m[2], m[3]);
        partial[3 * e + 1] = make_float4(m[4], m[5], m[6], m[7]);
        partial[3 * e + 2] = make_float4(m[8], m[9], 0.f, 0.f);
      } else {
        float* A = accum + (size_t)sg[j] * VACC;
#pragma unroll
        for (int k = 0; k < VACC; ++k) atomicAdd(A + k, m[k]);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_vox_bwd(const VoxArgs& a, bool det, const VoxRec* rec, const uint32_t* vals,
                           const uint32_t* emit_gid, const uint2* ranges, const float* dL_dV, float* accum,
                           float4* partial, cudaStream_t st) {
  int64_t tiles = (int64_t)a.TX * a.TY * a.TZ;
  if (tiles == 0) return cudaSuccess;
  if (det) k_vox_bwd<true><<<(unsigned)tiles, VNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dV, accum, partial);
  else k_vox_bwd<false><<<(unsigned)tiles, VNT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dV, accum, partial);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_vox_det_reduce(int n, const unsigned long long* __restrict__ offsets,
                                 const unsigned long long* __restrict__ counts, const float4* __restrict__ partial,
                                 float* __restrict__ accum) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float A[VACC];
#pragma unroll
  for (int k = 0; k < VACC; ++k) A[k] = 0.f;
  unsigned long long e0 = offsets[i], e1 = e0 + counts[i];
  for (unsigned long long e = e0; e < e1; ++e) {
    float4 p0 = partial[3 * e], p1 = partial[3 * e + 1], p2 = partial[3 * e + 2];
    A[0] += p0.x; A[1] += p0.y; A[2] += p0.z; A[3] += p0.w;
    A[4] += p1.x; A[5] += p1.y; A[6] += p1.z; A[7] += p1.w;
    A[8] += p2.x; A[9] += p2.y;
  }
#pragma unroll
  for (int k = 0; k < VACC; ++k) accum[(size_t)i * VACC + k] = A[k];
}

void launch_vox_det_reduce(int n, const unsigned long long* offsets, const unsigned long long* counts,
                           const float4* partial, float* accum, cudaStream_t st) {
  if (n <= 0) return;
  k_vox_det_reduce<<<ceil_div(n, 256), 256, 0, st>>>(n, offsets, counts, partial, accum);
  note_launch();
}

// Moments -> gradients:  dL/dalpha = M0,  dL/dmu = alpha K (M1, M2, M3),
// dL/dK (full matrix) = -1/2 alpha M_ij,  dL/dSigma = -K dL/dK K.
__global__ void __launch_bounds__(VPRE_THREADS) k_vox_bwd_pre(VoxArgs a, const float* __restrict__ accum,
                                                              float* __restrict__ d_mu, float* __restrict__ d_scale,
                                                              float* __restrict__ d_quat,
                                                              float* __restrict__ d_alpha) {
  int i = blockIdx.x * VPRE_THREADS + threadIdx.x;
  if (i >= a.n) return;
  float m[VACC];
#pragma unroll
  for (int k = 0; k < VACC; ++k) m[k] = accum[(size_t)i * VACC + k];
  float4 q = reinterpret_cast<const float4*>(a.quat)[i];
  float R[3][3], qn[4], qnorm;
  quat_rot(q, R, qn, qnorm);
  float dd[3] = {a.mod * a.scale[3 * i], a.mod * a.scale[3 * i + 1], a.mod * a.scale[3 * i + 2]};
  float M[3][3], Sw[6], K6[6];
  covariance(R, dd, M, Sw);
  float det = sym_inv3(Sw, K6);
  bool valid = det > 1e-30f && isfinite(det) && qnorm > 0.0f;
  float gmu[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, ga = 0.f;
  if (valid) {
    const float al = a.alpha[i];
    const float K[3][3] = {{K6[0], K6[1], K6[2]}, {K6[1], K6[3], K6[4]}, {K6[2], K6[4], K6[5]}};
    ga = m[0];
#pragma unroll
    for (int r = 0; r < 3; ++r) gmu[r] = al * (K[r][0] * m[1] + K[r][1] * m[2] + K[r][2] * m[3]);
    const float hm = -0.5f * al;
    const float GK[3][3] = {{hm * m[4], hm * m[7], hm * m[8]},
                            {hm * m[7], hm * m[5], hm * m[9]},
                            {hm * m[8], hm * m[9], hm * m[6]}};
    float T[3][3], Gw[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) T[r][c] = K[r][0] * GK[0][c] + K[r][1] * GK[1][c] + K[r][2] * GK[2][c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Gw[r][c] = -(T[r][0] * K[0][c] + T[r][1] * K[1][c] + T[r][2] * K[2][c]);
    scale_quat_backward(R, M, dd, qn, qnorm, a.mod, Gw, gs, gq);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d_mu[3 * i + k] = gmu[k];
    d_scale[3 * i + k] = gs[k];
  }
  reinterpret_cast<float4*>(d_quat)[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
  d_alpha[i] = ga;
}

// Algorithmic work of a voxelize: the voxel centres inside each Gaussian's
// culling ellipsoid d^T Sigma^-1 d <= 2 ln(1/eps), clipped to the grid.  One
// warp per Gaussian; each lane takes (y, z) rows of the bounding box and counts
// the row's x interval in closed form (double precision).  Added into *out.
__global__ void __launch_bounds__(256) k_vox_count(VoxArgs a, const VoxRec* __restrict__ rec,
                                                   unsigned long long* __restrict__ out) {
  const int g = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= a.n) return;
  const VoxRec r = rec[g];
  if (r.r3.y == 0.0f) return;
  const double mx = r.r0.x, my = r.r0.y, mz = r.r0.z;
  const double K00 = r.r1.x, K01 = r.r1.y, K02 = r.r1.z, K11 = r.r1.w, K12 = r.r2.x, K22 = r.r2.y;
  const double hy = r.r2.w, hz = r.r3.x, k2 = a.k2;
  const int y0 = max(0, (int)ceil(my - hy - 0.5)), y1 = min(a.Y - 1, (int)floor(my + hy - 0.5));
  const int z0 = max(0, (int)ceil(mz - hz - 0.5)), z1 = min(a.Z - 1, (int)floor(mz + hz - 0.5));
  unsigned long long cnt = 0;
  if (y1 >= y0 && z1 >= z0) {
    const int ny = y1 - y0 + 1;
    const int rows = ny * (z1 - z0 + 1);
    for (int i = lane; i < rows; i += 32) {
      const double dy = (y0 + i % ny) + 0.5 - my, dz = (z0 + i / ny) + 0.5 - mz;
      const double b = K01 * dy + K02 * dz;
      const double c = K11 * dy * dy + 2.0 * K12 * dy * dz + K22 * dz * dz;
      const double disc = b * b - K00 * (c - k2);
      if (disc < 0.0) continue;
      const double sq = sqrt(disc);
      const long long x0 = max(0LL, (long long)ceil(mx + (-b - sq) / K00 - 0.5));
      const long long x1 = min((long long)a.X - 1, (long long)floor(mx + (-b + sq) / K00 - 0.5));
      if (x1 >= x0) cnt += (unsigned long long)(x1 - x0 + 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0 && cnt) atomicAdd(out, cnt);
}

void launch_vox_count(const VoxArgs& a, const VoxRec* rec, unsigned long long* out, cudaStream_t st) {
  if (a.n <= 0) return;
  k_vox_count<<<ceil_div(a.n, 8), 256, 0, st>>>(a, rec, out);
  note_launch();
}

void launch_vox_bwd_pre(const VoxArgs& a, const float* accum, float* d_mu, float* d_scale, float* d_quat,
                        float* d_alpha, cudaStream_t st) {
  if (a.n <= 0) return;
  k_vox_bwd_pre<<<ceil_div(a.n, VPRE_THREADS), VPRE_THREADS, 0, st>>>(a, accum, d_mu, d_scale, d_quat, d_alpha);
  note_launch();
}

}  // namespace gp
