// voxel.cu -- sm_103a kernels of the differentiable voxelizer (GaussianPile,
// arXiv 2603.20611, Sec. 4.3 "Differentiable Voxelization", Eq. 12):
//     V(x) = sum_i alpha_i exp(-1/2 (x - mu_i)^T Sigma_i^-1 (x - mu_i))
// on a voxel grid partitioned into 8^3 tiles.
//
// Pipeline (the sort and scan are shared with the slice renderer):
//   K-vpre   per Gaussian: record (mu, alpha, K = Sigma^-1, bounding box of the
//            ellipsoid (x-mu)^T K (x-mu) <= 2 ln(1/eps)) + number of tiles
//   K-vemit  tile keys with emission indices
//   K-vfwd   one 64-thread CTA per tile; each warp owns an 8 x 4 x 8 half and
//            skips the Gaussians whose ellipsoid misses it (both shadows tested);
//            a lane owns a row of 8 voxels along x, whose exponent is a quadratic
//            in the x offset, two voxels per packed fp32x2 instruction
//   K-vbwd   one Gaussian per lane over the warp's half: ten moments
//            (sum G E, sum G E d_i, sum G E d_i d_j) from per-row sums, no
//            cross-lane reduction; the two halves summed in a fixed order, then
//            atomically added per Gaussian (or stored per pair for the
//            deterministic ordered reduction)
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

// Staging of one Gaussian for one 8^3 tile:
//   s0 = (mu - tile origin (x, y, z), alpha)
//   s1 = (q_xx, q_yy, q_zz, q_xy), s2 = (q_xz, q_yz): the exponent in base 2,
//        e = q_xx dx^2 + q_yy dy^2 + q_zz dz^2 + q_xy dx dy + q_xz dx dz + q_yz dy dz
//        = -log2(e)/2 d^T K d (off-diagonals doubled), K = Sigma^-1
//   h0 = (C00, C01, C11, 1/C00), h1 = (1/C11, D00, D01, D11), h2 = (1/D00, 1/D11):
//        the shadows of the culling ellipsoid on the xy plane (conic C, the Schur
//        complement of K_zz) and on the xz plane (conic D, the complement of K_yy).
struct VoxStage {
  float4 s0, s1, h0, h1;
  float4 s2h2;  // (q_xz, q_yz, 1/D00, 1/D11)
};

__device__ __forceinline__ VoxStage vstage(const VoxRec* __restrict__ rec, uint32_t g, float ox, float oy,
                                           float oz) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2);
  const float K00 = r1.x, K01 = r1.y, K02 = r1.z, K11 = r1.w, K12 = r2.x, K22 = r2.y;
  const float h = -0.5f * kLog2e;
  VoxStage v;
  v.s0 = make_float4(r0.x - ox, r0.y - oy, r0.z - oz, r0.w);
  v.s1 = make_float4(h * K00, h * K11, h * K22, 2.0f * h * K01);
  const float iz = 1.0f / K22, iy = 1.0f / K11;
  const float C00 = K00 - K02 * K02 * iz, C01 = K01 - K02 * K12 * iz, C11 = K11 - K12 * K12 * iz;
  const float D00 = K00 - K01 * K01 * iy, D01 = K02 - K01 * K12 * iy, D11 = K22 - K12 * K12 * iy;
  v.h0 = make_float4(C00, C01, C11, 1.0f / C00);
  v.h1 = make_float4(1.0f / C11, D00, D01, D11);
  v.s2h2 = make_float4(2.0f * h * K02, 2.0f * h * K12, 1.0f / D00, 1.0f / D11);
  return v;
}

// Does the culling ellipsoid reach the box [0.5, 7.5] x [y0, y1] x [0.5, 7.5]
// (voxel centres, tile-relative)?  Both of its shadows must reach the box's
// (conservative: an exact box test would cost a 3-D quadratic program).
__device__ __forceinline__ bool vox_box_hit(const VoxStage& v, float y0, float y1, float k2) {
  return ellipse_hits_rect(v.s0.x, v.s0.y, v.h0.x, v.h0.y, v.h0.z, v.h0.w, v.h1.x, k2, 0.5f, 7.5f, y0, y1) &&
         ellipse_hits_rect(v.s0.x, v.s0.z, v.h1.y, v.h1.z, v.h1.w, v.s2h2.z, v.s2h2.w, k2, 0.5f, 7.5f, 0.5f, 7.5f);
}

// Row coefficients along x for the row (dy, dz): e = A + B q + C q^2 with
// q = x - 4 the offset from the tile's centre column and dxc = 4 - mu_x.
__device__ __forceinline__ void vrow(const float4& s1, float qxz, float qyz, float dxc, float dy, float dz, float& A,
                                     float& B) {
  const float lin = fmaf(s1.w, dy, qxz * dz);  // q_xy dy + q_xz dz
  B = fmaf(2.0f * s1.x, dxc, lin);
  A = fmaf(dxc, fmaf(s1.x, dxc, lin), fmaf(s1.y * dy, dy, fmaf(s1.z * dz, dz, qyz * dy * dz)));
}

struct VoxFwdSmem {
  VoxStage st[VCH];
  int hits[VNT / 32][VCH];
};

// Forward: one 64-thread CTA per 8^3 tile; warp w owns the 8 x 4 x 8 half with
// y in [4w, 4w + 4); lane (yl, z) owns the row of 8 voxels along x at y = 4w + yl
// and z, two voxels per packed instruction.  Each staged Gaussian is tested
// against the warp's half (its xy and xz shadows), and the hits are applied in
// chunk order (bitwise reproducible sums).
template <int EXPM>
__global__ void __launch_bounds__(VNT) k_vox_fwd(VoxArgs a, const VoxRec* __restrict__ rec,
                                                 const uint32_t* __restrict__ vals,
                                                 const uint32_t* __restrict__ emit_gid,
                                                 const uint2* __restrict__ ranges, float* __restrict__ vol) {
  __shared__ VoxFwdSmem sm;
  const int tile = blockIdx.x;
  const int tx = tile % a.TX, ty = (tile / a.TX) % a.TY, tz = tile / (a.TX * a.TY);
  const uint2 rg = ranges[tile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int yl = lane & 3, zl = lane >> 2;
  const float ox = (float)(tx * VOX_TILE), oy = (float)(ty * VOX_TILE), oz = (float)(tz * VOX_TILE);
  const float py = (float)(4 * warp + yl) + 0.5f, pz = (float)zl + 0.5f;
  const float y0 = (float)(4 * warp) + 0.5f;
  int* hits = sm.hits[warp];
  float2 acc[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) acc[p] = make_float2(0.f, 0.f);
  for (uint32_t base = rg.x; base < rg.y; base += VCH) {
    const int cnt = (int)min((uint32_t)VCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += VNT) sm.st[j] = vstage(rec, emit_gid[vals[base + j]], ox, oy, oz);
    __syncthreads();
    int nh = 0;
    for (int jb = 0; jb < cnt; jb += 32) {
      const int j = jb + lane;
      const bool hit = j < cnt && vox_box_hit(sm.st[j], y0, y0 + 3.0f, a.k2);
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) hits[nh + __popc(m & ((1u << lane) - 1u))] = j;
      nh += __popc(m);
    }
    __syncwarp();
    for (int h = 0; h < nh; ++h) {
      const VoxStage& v = sm.st[hits[h]];
      const float4 g0 = v.s0, g1 = v.s1;
      float A, B;
      vrow(g1, v.s2h2.x, v.s2h2.y, 4.0f - g0.x, py - g0.y, pz - g0.z, A, B);
      const float2 C2 = make_float2(g1.x, g1.x), B2 = make_float2(B, B), A2 = make_float2(A, A);
      const float2 al2 = make_float2(g0.w, g0.w);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float2 q = make_float2((float)(2 * p) - 3.5f, (float)(2 * p + 1) - 3.5f);
        acc[p] = __ffma2_rn(al2, pair_exp2<EXPM>(C2, B2, A2, q), acc[p]);
      }
    }
    __syncthreads();
  }
  const int y = ty * VOX_TILE + 4 * warp + yl, z = tz * VOX_TILE + zl;
  if (y < a.Y && z < a.Z) {
    float* o = vol + ((int64_t)z * a.Y + y) * a.X + tx * VOX_TILE;
    const int xr = a.X - tx * VOX_TILE;  // voxels of this row inside the volume
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (2 * p < xr) o[2 * p] = acc[p].x;
      if (2 * p + 1 < xr) o[2 * p + 1] = acc[p].y;
    }
  }
}

cudaError_t launch_vox_fwd(const VoxArgs& a, const VoxRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                           const uint2* ranges, float* vol, cudaStream_t st) {
  int64_t tiles = (int64_t)a.TX * a.TY * a.TZ;
  if (tiles == 0) return cudaSuccess;
  k_vox_fwd<GP_EXP_POLY><<<(unsigned)tiles, VNT, 0, st>>>(a, rec, vals, emit_gid, ranges, vol);
  note_launch();
  return cudaGetLastError();
}

struct VoxBwdSmem {
  VoxStage st[VCH];
  uint32_t sg[VCH];
  alignas(16) float G[VOX_TILE][VOX_TILE][VOX_TILE];  // the tile's dL/dV [z][y][x], zero outside the volume
  int hits[VNT / 32][VCH];
  unsigned hmask[VNT / 32][VCH / 32];
  float sp[VNT / 32][VACC][VCH];
};

// Backward: warp w owns the same 8 x 4 x 8 half as in the forward.  Each lane
// takes one hit Gaussian at a time and sums, over the half's 128 voxels (16 rows
// of 8 along x, two voxels per packed instruction, dL/dV read from shared memory
// as broadcasts), the ten moments
//     sum G E {1, dx, dy, dz, dx^2, dy^2, dz^2, dx dy, dx dz, dy dz}
// (E the Gaussian's exponential, G = dL/dV, d = voxel - mu) from per-row sums
// about the centre column; no lane shares a Gaussian, so nothing is reduced
// across lanes.  The two halves' moments are added in a fixed order and folded
// into the Gaussian's accumulators (atomics) or a per-pair partial.
template <bool DET>
__global__ void __launch_bounds__(VNT) k_vox_bwd(VoxArgs a, const VoxRec* __restrict__ rec,
                                                 const uint32_t* __restrict__ vals,
                                                 const uint32_t* __restrict__ emit_gid,
                                                 const uint2* __restrict__ ranges, const float* __restrict__ dL_dV,
                                                 float* __restrict__ accum, float4* __restrict__ partial) {
  constexpr int NW = VNT / 32;
  __shared__ VoxBwdSmem sm;
  const int tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  if (rg.y <= rg.x) return;  // uniform over the CTA
  const int tx = tile % a.TX, ty = (tile / a.TX) % a.TY, tz = tile / (a.TX * a.TY);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float ox = (float)(tx * VOX_TILE), oy = (float)(ty * VOX_TILE), oz = (float)(tz * VOX_TILE);
  const float y0 = (float)(4 * warp) + 0.5f;
  for (int i = threadIdx.x; i < VOX_TILE * VOX_TILE * VOX_TILE; i += VNT) {
    const int xx = i & 7, yy = (i >> 3) & 7, zz = i >> 6;
    const int x = tx * VOX_TILE + xx, y = ty * VOX_TILE + yy, z = tz * VOX_TILE + zz;
    sm.G[zz][yy][xx] = (x < a.X && y < a.Y && z < a.Z) ? dL_dV[((int64_t)z * a.Y + y) * a.X + x] : 0.f;
  }
  int* hits = sm.hits[warp];
  for (uint32_t base = rg.x; base < rg.y; base += VCH) {
    const int cnt = (int)min((uint32_t)VCH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += VNT) {
      const uint32_t g = emit_gid[vals[base + j]];
      sm.st[j] = vstage(rec, g, ox, oy, oz);
      sm.sg[j] = g;
    }
    __syncthreads();
    int nh = 0;
    for (int jb = 0; jb < VCH; jb += 32) {
      const int j = jb + lane;
      const bool hit = j < cnt && vox_box_hit(sm.st[j], y0, y0 + 3.0f, a.k2);
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) hits[nh + __popc(m & ((1u << lane) - 1u))] = j;
      if (lane == 0) sm.hmask[warp][jb >> 5] = m;
      nh += __popc(m);
    }
    __syncwarp();
    for (int u0 = 0; u0 < nh; u0 += 32) {
      const int u = u0 + lane;
      if (u >= nh) break;
      const int jj = hits[u];
      const VoxStage& v = sm.st[jj];
      const float4 g0 = v.s0, g1 = v.s1;
      const float dxc = 4.0f - g0.x;
      const float2 C2 = make_float2(g1.x, g1.x);
      float T0 = 0.f, T1 = 0.f, T2 = 0.f, Y0 = 0.f, Y1 = 0.f, Z0 = 0.f, Z1 = 0.f, YY = 0.f, ZZ = 0.f, YZ = 0.f;
      for (int zz = 0; zz < VOX_TILE; ++zz) {
        const float dz = ((float)zz + 0.5f) - g0.z;
#pragma unroll
        for (int yl = 0; yl < 4; ++yl) {
          const float dy = (float)(4 * warp + yl) + 0.5f - g0.y;
          float A, B;
          vrow(g1, v.s2h2.x, v.s2h2.y, dxc, dy, dz, A, B);
          const float2 A2 = make_float2(A, A), B2 = make_float2(B, B);
          const float4 ga = *reinterpret_cast<const float4*>(&sm.G[zz][4 * warp + yl][0]);
          const float4 gb = *reinterpret_cast<const float4*>(&sm.G[zz][4 * warp + yl][4]);
          const float2 Gp[4] = {make_float2(ga.x, ga.y), make_float2(ga.z, ga.w), make_float2(gb.x, gb.y),
                                make_float2(gb.z, gb.w)};
          float2 P0 = make_float2(0.f, 0.f), P1 = P0, P2 = P0;
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float qa = (float)(2 * p) - 3.5f, qb = (float)(2 * p + 1) - 3.5f;
            const float2 q = make_float2(qa, qb);
            const float2 gE = __fmul2_rn(Gp[p], pair_exp2<GP_EXP_POLY>(C2, B2, A2, q));
            P0 = __fadd2_rn(P0, gE);
            P1 = __ffma2_rn(q, gE, P1);
            P2 = __ffma2_rn(make_float2(qa * qa, qb * qb), gE, P2);
          }
          const float S0 = P0.x + P0.y, S1 = P1.x + P1.y, S2 = P2.x + P2.y;
          T0 += S0;
          T1 += S1;
          T2 += S2;
          Y0 = fmaf(dy, S0, Y0);
          Y1 = fmaf(dy, S1, Y1);
          Z0 = fmaf(dz, S0, Z0);
          Z1 = fmaf(dz, S1, Z1);
          YY = fmaf(dy * dy, S0, YY);
          ZZ = fmaf(dz * dz, S0, ZZ);
          YZ = fmaf(dy * dz, S0, YZ);
        }
      }
      // moments in d = (dxc + q, dy, dz)
      float* sp = &sm.sp[warp][0][jj];
      sp[0 * VCH] = T0;
      sp[1 * VCH] = fmaf(dxc, T0, T1);
      sp[2 * VCH] = Y0;
      sp[3 * VCH] = Z0;
      sp[4 * VCH] = fmaf(dxc, fmaf(dxc, T0, 2.0f * T1), T2);
      sp[5 * VCH] = YY;
      sp[6 * VCH] = ZZ;
      sp[7 * VCH] = fmaf(dxc, Y0, Y1);
      sp[8 * VCH] = fmaf(dxc, Z0, Z1);
      sp[9 * VCH] = YZ;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += VNT) {
      float m[VACC];
#pragma unroll
      for (int k = 0; k < VACC; ++k) m[k] = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w)
        if ((sm.hmask[w][j >> 5] >> (j & 31)) & 1u) {
#pragma unroll
          for (int k = 0; k < VACC; ++k) m[k] += sm.sp[w][k][j];
        }
      if constexpr (DET) {
        const size_t e = vals[base + j];
        partial[3 * e] = make_float4(m[0], m[1], m[2], m[3]);
        partial[3 * e + 1] = make_float4(m[4], m[5], m[6], m[7]);
        partial[3 * e + 2] = make_float4(m[8], m[9], 0.f, 0.f);
      } else {
        float* A = accum + (size_t)sm.sg[j] * VACC;
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
