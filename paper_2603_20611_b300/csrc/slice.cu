// slice.cu -- sm_103a kernels of the finite-thickness slice projection operator
// (GaussianPile, arXiv 2603.20611, Sec. 4.2 Eq. 6-10 forward, Sec. 4.3 backward).
//
// Closed form used on the device.  In the camera frame of the view [R_c | t]
// (Sec. S1: mu_c = R_c mu + t, Sigma_c = R_c Sigma R_c^T; R_c an axis
// permutation or any rotation shared by the stack's planes), with slice axis c,
// in-plane axes p and a plane at z_s, the paper's inverse-covariance update (Eq. 6), opacity
// modulation (Eq. 7) and marginal (Eq. 8) reduce, by the Sherman-Morrison
// identity, to
//     v = Sigma_cc + sigma_z^2,  a = Sigma_pc / v,
//     Sigma_2d = Sigma_pp - Sigma_pc Sigma_cp / v,                 (slice-invariant)
//     mu_2d = mu_p - a delta,  opacity_r = exp(-delta^2 / 2v),     delta = mu_c - z_s,
// and a~ = alpha opacity_r / sqrt(det Sigma_2d) (Eq. 9).  So one 64-byte record
// per Gaussian (K-pre) serves every slice; per (Gaussian, slice) only mu_2d and
// a~ change, and each Gaussian touches a contiguous run of planes
// |delta| <= sqrt(2 v ln(1/eps)).
//
// Pipeline of one render:
//   K-pre     per Gaussian: record + number of (slice, tile) pairs it touches
//             (a warp per 32 Gaussians, their work dealt out by plane and by
//             tile row)
//   scan      exclusive scan of the counts (sort.cu)
//   K-emit    keys (slice * T + tile) with Gaussian ids as values, in Gaussian
//             order (the same warp-balanced enumeration)
//   sort      stable one-sweep radix sort on the live key bits (sort.cu)
//   K-range   [start, end) of every (slice, tile)
//   K-fwd     one CTA per (slice, tile): stage the tile's Gaussians in shared
//             memory with 16-byte loads, every thread accumulates PX pixels of
//             a row (Eq. 10)
// Backward (no per-pixel state is stored; lists are rebuilt):
//   K-bwd     per (slice, tile): recompute each exponential, form six pixel
//             moments per Gaussian, warp-shuffle reduce them, combine the warps
//             in a fixed order, then either atomically fold them into ten
//             per-Gaussian accumulators or write per-pair partials
//   K-det     (deterministic mode) ordered per-Gaussian reduction of partials
//   K-bwd-pre accumulators -> dL/d(mu, scale, quat, alpha) in closed form
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gp_check.cuh"
#include "gp_common.cuh"
#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

constexpr int PRE_THREADS = 128;

// ------------------------------------------------------------ K-pre
__device__ __forceinline__ int lower_bound_f(const float* __restrict__ v, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (v[m] < x) lo = m + 1; else hi = m;
  }
  return lo;
}

__device__ __forceinline__ int upper_bound_f(const float* __restrict__ v, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (v[m] <= x) lo = m + 1; else hi = m;
  }
  return lo;
}

// 1 / tile for the power-of-two tile sides (exact, without a division).
__device__ __forceinline__ float tile_rcp(int tile) { return tile == 8 ? 0.125f : 0.0625f; }

__device__ __forceinline__ int clamp_tile(float t, int nt) {
  // t is a (possibly huge) tile coordinate; clamp in float first
  t = fminf(fmaxf(t, -1.0f), (float)nt);
  return (int)floorf(t);
}

// Visits every (sorted slice position j, tile) pair of one Gaussian: planes with
// |mu_z - z_s| <= zr, tiles whose pixel-centre rectangle the ellipse
// d^T C d <= k2 around mu_2d touches.  Arithmetic uses explicit rounding so every
// caller takes identical decisions.
// Planes of one Gaussian: sorted positions [lo, hi) with |mu_z - z_s| <= zr.
__device__ __forceinline__ void plane_range(const SliceArgs& a, const SliceRec& r, int& lo, int& hi) {
  const float mz = r.r0.z, zr = r.r1.w;
  lo = lower_bound_f(a.zs, a.S, __fsub_rn(mz, zr));
  hi = upper_bound_f(a.zs, a.S, __fadd_rn(mz, zr));
}

// mu_2d on sorted plane j, the culling ellipse on it and the clamped range of
// tile rows the ellipse spans.  On a slice the ellipse is d^T C d <= k2 on every
// plane the pair reaches; on a voxelizer plane the cut is the 3D one,
// d^T C d + delta^2 / Sigma_zz <= k2, so the plane's ellipse is d^T C d <= k2 -
// delta^2 / Sigma_zz, its half-extents rx, ry scaled by sqrt(k2e / k2).
struct PlaneBox {
  float mx, my;
  float k2e, rxe, rye;  // the plane's squared radius and half-extents
  int ty0, ty1;
};

__device__ __forceinline__ PlaneBox plane_box(const SliceArgs& a, const SliceRec& r, int j) {
  PlaneBox b;
  const float inv_tile = tile_rcp(a.tile);
  const float d = __fsub_rn(r.r0.z, a.zs[j]);
  b.k2e = a.k2;
  b.rxe = r.r2.w;
  b.rye = r.r3.x;
  if (a.vox) {
    b.k2e = fmaxf(__fsub_rn(a.k2, __fmul_rn(__fmul_rn(d, d), r.r0.w)), 0.0f);
    const float f = __fsqrt_rn(__fdiv_rn(b.k2e, a.k2));
    b.rxe = __fmul_rn(b.rxe, f);
    b.rye = __fmul_rn(b.rye, f);
  }
  const float ry = b.rye;
  b.mx = __fsub_rn(r.r0.x, __fmul_rn(r.r1.x, d));
  b.my = __fsub_rn(r.r0.y, __fmul_rn(r.r1.y, d));
  b.ty0 = max(0, clamp_tile(__fmul_rn(__fsub_rn(__fsub_rn(b.my, ry), 0.5f), inv_tile), a.TY));
  b.ty1 = min(a.TY - 1, clamp_tile(__fmul_rn(__fsub_rn(__fadd_rn(b.my, ry), 0.5f), inv_tile), a.TY));
  return b;
}

// Tile columns [*lo, *hi] of tile row ty whose pixel-centre rectangle the ellipse
// d^T C d <= k2 touches.  Over the row's band of pixel-centre heights the ellipse
// spans x in [xmin, xmax]: with s = C01/C00 and D = C11 - C01 s, the chord at
// height dy is centred on -s dy with half-width sqrt((k2 - D dy^2)/C00), and its
// right (left) end is largest (smallest) at the tangent height dy_t = -C01 rx/C11
// (-dy_t), clamped to the band.  A tile is touched iff its x-range meets
// [xmin, xmax].  Explicit roundings keep the count and the emission identical.
__device__ __forceinline__ bool row_tiles(const SliceArgs& a, const SliceRec& r, const PlaneBox& b, int ty,
                                          int* lo, int* hi) {
  const float c01 = r.r2.y, c11 = r.r2.z, rx = b.rxe, ry = b.rye, k2 = b.k2e;
  const float inv00 = r.r3.z, inv11 = r.r3.w;
  const float y0 = (float)(ty * a.tile) + 0.5f;
  const float y1 = (float)(min((ty + 1) * a.tile, a.H)) - 0.5f;
  const float dya = fmaxf(__fsub_rn(y0, b.my), -ry);
  const float dyb = fminf(__fsub_rn(y1, b.my), ry);
  if (dya > dyb) return false;
  const float s = __fmul_rn(c01, inv00);
  const float D = __fsub_rn(c11, __fmul_rn(c01, s));
  const float dyt = -__fmul_rn(__fmul_rn(c01, inv11), rx);
  const float dM = fminf(fmaxf(dyt, dya), dyb);
  const float dm = fminf(fmaxf(-dyt, dya), dyb);
  const float wM = __fsqrt_rn(fmaxf(__fmul_rn(__fsub_rn(k2, __fmul_rn(D, __fmul_rn(dM, dM))), inv00), 0.0f));
  const float wm = __fsqrt_rn(fmaxf(__fmul_rn(__fsub_rn(k2, __fmul_rn(D, __fmul_rn(dm, dm))), inv00), 0.0f));
  const float xmax = __fadd_rn(__fsub_rn(b.mx, __fmul_rn(s, dM)), wM);
  const float xmin = __fsub_rn(__fsub_rn(b.mx, __fmul_rn(s, dm)), wm);
  const float inv_tile = tile_rcp(a.tile);
  // tile tx spans pixel centres [tx T + 0.5, (tx + 1) T - 0.5] (the last one ends at W - 0.5)
  int l = max(0, clamp_tile(__fmul_rn(__fadd_rn(xmin, 0.5f), inv_tile), a.TX + 1) - 1);
  const float lf = __fsub_rn(__fmul_rn(__fadd_rn(xmin, 0.5f), inv_tile), 1.0f);
  if ((float)l < lf) l += 1;  // ceil of (xmin + 0.5)/T - 1
  int h = min(a.TX - 1, clamp_tile(__fmul_rn(__fsub_rn(xmax, 0.5f), inv_tile), a.TX));
  if (h == a.TX - 1 && xmin > (float)a.W - 0.5f) h = a.TX - 2;
  *lo = l;
  *hi = h;
  return h >= l;
}

template <class F>
__device__ __forceinline__ void for_each_pair(const SliceArgs& a, const SliceRec& r, F&& f) {
  if (r.r3.y == 0.0f) return;
  int plo, phi;
  plane_range(a, r, plo, phi);
  for (int j = plo; j < phi; ++j) {
    const PlaneBox b = plane_box(a, r, j);
    for (int ty = b.ty0; ty <= b.ty1; ++ty) {
      int lo, hi;
      if (!row_tiles(a, r, b, ty, &lo, &hi)) continue;
      for (int tx = lo; tx <= hi; ++tx)
        if (GP_IN_RANGE(7, tx, a.TX) && GP_IN_RANGE(8, ty, a.TY)) f(j, ty * a.TX + tx);
    }
  }
}

// Record of Gaussian i of item a.
__device__ __forceinline__ SliceRec make_record(const SliceArgs& a, int i) {
  float4 q = reinterpret_cast<const float4*>(a.quat)[i];
  float R[3][3], qn[4], qnorm;
  quat_rot(q, R, qn, qnorm);
  float d3[3] = {a.mod * a.scale[3 * i], a.mod * a.scale[3 * i + 1], a.mod * a.scale[3 * i + 2]};
  float M[3][3], Sw[6];
  covariance(R, d3, M, Sw);
  // camera frame of the view: mu_c = R_c mu + t, Sigma_c = R_c Sigma R_c^T
  float mc[3], Sc[6];
  camera_frame(a.Rc, a.tc, a.mu + 3 * i, Sw, mc, Sc);
  float cxx = Sc[0], cxy = Sc[1], cxz = Sc[2], cyy = Sc[3], cyz = Sc[4], czz = Sc[5];
  float mux = mc[0], muy = mc[1], muz = mc[2];
  float v = czz + a.sigma2;
  float iv = 1.0f / v;
  float ax = cxz * iv, ay = cyz * iv;
  float sxx = cxx - cxz * ax, sxy = cxy - cxz * ay, syy = cyy - cyz * ay;
  float det = sxx * syy - sxy * sxy;
  bool valid = det > 1e-30f && isfinite(det) && isfinite(v) && isfinite(mux) && isfinite(muy) &&
               isfinite(muz) && qnorm > 0.0f && isfinite(a.alpha[i]);
  float idet = 1.0f / det;
  SliceRec r;
  r.r0 = make_float4(mux, muy, muz, iv);
  // amplitude: alpha / sqrt(det Sigma_2d) on a slice (Eq. 9); alpha on a voxelizer plane, where the
  // Gaussian on the plane z is alpha exp(-delta^2 / 2 Sigma_zz) exp(-d^T Sigma_2d^-1 d / 2) (Eq. 12)
  r.r1 = make_float4(ax, ay, a.vox ? a.alpha[i] : a.alpha[i] / sqrtf(det), sqrtf(a.k2 * v));
  r.r2 = make_float4(syy * idet, -sxy * idet, sxx * idet, sqrtf(a.k2 * sxx));
  r.r3 = make_float4(sqrtf(a.k2 * syy), valid ? 1.0f : 0.0f, det / syy, det / sxx);
  return r;
}

// Item owning batch-wide index x of a prefix table t[0..n] (t[0] = 0).
template <typename T>
__device__ __forceinline__ int find_item(const T* __restrict__ t, int n, T x) {
  int lo = 0, hi = n;  // invariant: t[lo] <= x < t[hi]
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (t[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

// ------------------------------------------------------------ K-pre / K-emit
// Both are warp-balanced.  With a thread per Gaussian a warp waits for its
// largest Gaussian: on the microscopy fit step (500k Gaussians, 16 of 256
// planes) a warp's largest Gaussian has 3.7x the mean pair count and 3.0x the
// mean number of tile rows.  Here a warp takes 32 consecutive Gaussians and
// deals their work out in two stages: the (Gaussian, plane) items 32 at a
// time, then those items' tile rows 32 at a time, each lane finding its item
// (row) by a binary search over the warp's prefix counts in shared memory.
// K-pre adds each row's tile count to its Gaussian's count; K-emit places each
// row's pairs by a warp scan of the row counts, so the pairs leave in the order
// of for_each_pair (Gaussian, plane, tile row, tile column) and the counts and
// the emission agree by construction.
constexpr int BAL_WARPS = 4;

template <bool EMIT>
struct BalSmem {
  SliceRec rec[32];  // the warp's records
  int item0[33];     // exclusive prefix of the lanes' plane counts
  int plo[32];       // each lane's first sorted plane
  int row0[33];      // exclusive prefix of the current items' tile-row counts
  int owner[32], ty0[32];
  float mx[32], my[32], k2e[32], rxe[32], rye[32];
  unsigned cnt[32];  // K-pre: pairs of each lane's Gaussian
  int iown[32];      // the lane owning each item of the current round
  int rown[32];      // the item slot owning each tile row of the current round
  uint32_t kb[32];    // K-emit: the key of each current item's plane and tile (0, 0)
};

// Marks the slots [c0, c0 + 32) of a round that this lane's run [b, e) of a
// warp-wide sequence covers with the lane's index (each slot is covered by
// exactly one lane), so that a lane finds the owner of its slot with one load.
__device__ __forceinline__ void bal_mark(int* own, int b, int e, int c0, int lane) {
  const int s = max(b, c0) - c0, t = min(e, c0 + 32) - c0;
  for (int p = s; p < t; ++p) own[p] = lane;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// One warp over the Gaussians of one item whose batch-wide indices are
// i0 + [lane_lo, lane_hi) (local index = batch-wide index - gbase0).  K-pre
// (EMIT false): make the records, store them and the pair counts.  K-emit (EMIT
// true): read the records and write the pairs (keys and batch-wide Gaussian
// ids) from index e0 on, never at or past e_end.
template <bool EMIT>
__device__ __forceinline__ void bal_warp(const SliceArgs& a, int i0, int lane_lo, int lane_hi, int gbase0,
                                         BalSmem<EMIT>& sm, SliceRec* __restrict__ rec,
                                         unsigned long long* __restrict__ counts, unsigned long long e0,
                                         unsigned long long e_end, uint32_t* __restrict__ keys,
                                         uint32_t* __restrict__ emit_gid) {
  const int lane = threadIdx.x & 31;
  const int i = i0 + lane;
  const bool live = lane >= lane_lo && lane < lane_hi;
  SliceRec r{};
  if (live) {
    if (EMIT) {
      r = rec[i];
    } else {
      r = make_record(a, i - gbase0);
      rec[i] = r;
    }
  }
  int plo = 0, phi = 0;
  if (live && r.r3.y != 0.0f) plane_range(a, r, plo, phi);
  sm.rec[lane] = r;
  sm.plo[lane] = plo;
  const int iincl = warp_incl_scan(phi - plo, lane), iexcl = iincl - (phi - plo);
  sm.item0[lane + 1] = iincl;
  if (lane == 0) sm.item0[0] = 0;
  if (!EMIT) sm.cnt[lane] = 0u;
  const int n_items = __shfl_sync(0xffffffffu, iincl, 31);
  const uint32_t T = (uint32_t)(a.TX * a.TY);
  __syncwarp();
  for (int c0 = 0; c0 < n_items; c0 += 32) {
    const int k = c0 + lane;
    int ny = 0;
    bal_mark(sm.iown, iexcl, iincl, c0, lane);
    __syncwarp();
    if (k < n_items) {
      const int o = sm.iown[lane];
      const int j = sm.plo[o] + (k - sm.item0[o]);
      const PlaneBox b = plane_box(a, sm.rec[o], j);
      ny = max(b.ty1 - b.ty0 + 1, 0);
      sm.owner[lane] = o;
      if (EMIT) sm.kb[lane] = a.key_base + (uint32_t)a.zorder[j] * T;
      sm.ty0[lane] = b.ty0;
      sm.mx[lane] = b.mx;
      sm.my[lane] = b.my;
      sm.k2e[lane] = b.k2e;
      sm.rxe[lane] = b.rxe;
      sm.rye[lane] = b.rye;
    }
    const int rincl = warp_incl_scan(ny, lane);
    sm.row0[lane + 1] = rincl;
    if (lane == 0) sm.row0[0] = 0;
    const int n_rows = __shfl_sync(0xffffffffu, rincl, 31);
    for (int q0 = 0; q0 < n_rows; q0 += 32) {
      const int q = q0 + lane;
      int lo = 0, hi = -1, o = 0, m = 0, ty = 0;
      __syncwarp();  // the last round's owners are read
      bal_mark(sm.rown, rincl - ny, rincl, q0, lane);
      __syncwarp();
      if (q < n_rows) {
        m = sm.rown[lane];
        o = sm.owner[m];
        ty = sm.ty0[m] + (q - sm.row0[m]);
        PlaneBox b;
        b.mx = sm.mx[m];
        b.my = sm.my[m];
        b.k2e = sm.k2e[m];
        b.rxe = sm.rxe[m];
        b.rye = sm.rye[m];
        if (!row_tiles(a, sm.rec[o], b, ty, &lo, &hi)) {
          lo = 0;
          hi = -1;
        }
      }
      const int c = hi - lo + 1;  // pairs of this tile row (0 if none)
      if (!EMIT) {
        if (c > 0) atomicAdd(&sm.cnt[o], (unsigned)c);
      } else {
        const int cincl = warp_incl_scan(c, lane);
        unsigned long long e = e0 + (unsigned long long)(cincl - c);
        if (c > 0) {
          const uint32_t kb = sm.kb[m] + (uint32_t)(ty * a.TX);
          const uint32_t gid = (uint32_t)(i0 + o);
          for (int tx = lo; tx <= hi; ++tx, ++e) {
            if (e < e_end && GP_IN_RANGE(7, tx, a.TX) && GP_IN_RANGE(8, ty, a.TY)) {
              keys[e] = kb + (uint32_t)tx;
              emit_gid[e] = gid;
            }
          }
        }
        e0 += (unsigned long long)__shfl_sync(0xffffffffu, cincl, 31);
      }
    }
    __syncwarp();  // the next items overwrite this round's item arrays
  }
  if (!EMIT && live) counts[i] = sm.cnt[lane];
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// The warp's pair counts: K-pre's per-warp total (wsum) after the warp's
// bal_warp calls have written its lanes' counts, or K-emit's placement from
// the scan of those totals (wsum = their exclusive scan): each Gaussian's
// offset (written out, the deterministic backward reads them) and a lane
// range's run [e0, e_end) of the output.
struct WarpRun {
  unsigned long long base, incl, cnt;
};

template <bool EMIT>
__device__ __forceinline__ WarpRun warp_run(const unsigned long long* __restrict__ counts,
                                            unsigned long long* __restrict__ wsum,
                                            unsigned long long* __restrict__ offsets, int wg, int i0, int nl,
                                            int lane) {
  WarpRun w{0ull, 0ull, 0ull};
  if (EMIT) {
    w.cnt = lane < nl ? counts[i0 + lane] : 0ull;
    w.incl = warp_incl_scan_u64(w.cnt, lane);
    w.base = wsum[wg];
    if (lane < nl) offsets[i0 + lane] = w.base + w.incl - w.cnt;
  }
  return w;
}

__device__ __forceinline__ void warp_total(const unsigned long long* __restrict__ counts,
                                           unsigned long long* __restrict__ wsum, int wg, int i0, int nl,
                                           int lane) {
  unsigned long long c = lane < nl ? counts[i0 + lane] : 0ull;  // this lane's own store
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) wsum[wg] = c;
}

template <bool EMIT>
__global__ void __launch_bounds__(BAL_WARPS * 32) k_slice_bal(SliceArgs a, SliceRec* __restrict__ rec,
                                                              unsigned long long* __restrict__ counts,
                                                              unsigned long long* __restrict__ wsum,
                                                              unsigned long long* __restrict__ offsets,
                                                              unsigned long long cap,
                                                              uint32_t* __restrict__ keys,
                                                              uint32_t* __restrict__ emit_gid) {
  __shared__ BalSmem<EMIT> sm[BAL_WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * BAL_WARPS + w;
  const int i0 = wg * 32;
  if (i0 >= a.n) return;  // uniform over the warp
  const int nl = min(32, a.n - i0);
  const WarpRun wr = warp_run<EMIT>(counts, wsum, offsets, wg, i0, nl, lane);
  const unsigned long long end = __shfl_sync(0xffffffffu, wr.incl, 31);
  bal_warp<EMIT>(a, i0, 0, nl, 0, sm[w], rec, counts, wr.base, min(wr.base + end, cap), keys, emit_gid);
  if (!EMIT) warp_total(counts, wsum, wg, i0, nl, lane);
}

// Batched form: the warp's 32 batch-wide Gaussians, one item at a time (items
// own contiguous ranges of Gaussians, so each one's share is a lane range).
template <bool EMIT>
__global__ void __launch_bounds__(BAL_WARPS * 32) k_slice_bal_batch(BatchItems b, SliceRec* __restrict__ rec,
                                                                    unsigned long long* __restrict__ counts,
                                                                    unsigned long long* __restrict__ wsum,
                                                                    unsigned long long* __restrict__ offsets,
                                                                    unsigned long long cap,
                                                                    uint32_t* __restrict__ keys,
                                                                    uint32_t* __restrict__ emit_gid) {
  __shared__ BalSmem<EMIT> sm[BAL_WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * BAL_WARPS + w;
  const int i0 = wg * 32;
  if (i0 >= b.n_gauss) return;  // uniform over the warp
  const int nl = min(32, b.n_gauss - i0);
  const WarpRun wr = warp_run<EMIT>(counts, wsum, offsets, wg, i0, nl, lane);
  for (int l = 0; l < nl;) {  // uniform over the warp
    const int k = find_item(b.gstart, b.n_items, i0 + l);
    const int g0 = b.gstart[k];
    const int lh = min(nl, b.gstart[k + 1] - i0);
    const SliceArgs a = b.args[k];
    const unsigned long long e0 = wr.base + __shfl_sync(0xffffffffu, wr.incl - wr.cnt, l);
    const unsigned long long e1 = wr.base + __shfl_sync(0xffffffffu, wr.incl, lh - 1);
    bal_warp<EMIT>(a, i0, l, lh, g0, sm[w], rec, counts, e0, min(e1, cap), keys, emit_gid);
    __syncwarp();
    l = lh;
  }
  if (!EMIT) warp_total(counts, wsum, wg, i0, nl, lane);
}

void launch_slice_pre(const SliceArgs& a, SliceRec* rec, unsigned long long* counts, unsigned long long* wsum,
                      cudaStream_t st) {
  if (a.n <= 0) return;
  k_slice_bal<false><<<ceil_div(a.n, BAL_WARPS * 32), BAL_WARPS * 32, 0, st>>>(a, rec, counts, wsum, nullptr, 0ull,
                                                                               nullptr, nullptr);
  note_launch();
}

void launch_slice_pre_batch(const BatchItems& b, SliceRec* rec, unsigned long long* counts, unsigned long long* wsum,
                            cudaStream_t st) {
  if (b.n_gauss <= 0) return;
  k_slice_bal_batch<false><<<ceil_div(b.n_gauss, BAL_WARPS * 32), BAL_WARPS * 32, 0, st>>>(
      b, rec, counts, wsum, nullptr, 0ull, nullptr, nullptr);
  note_launch();
}

void launch_slice_emit(const SliceArgs& a, const SliceRec* rec, const unsigned long long* woff,
                       const unsigned long long* counts, unsigned long long* offsets, uint32_t* keys,
                       uint32_t* emit_gid, cudaStream_t st, unsigned long long cap) {
  if (a.n <= 0) return;
  k_slice_bal<true><<<ceil_div(a.n, BAL_WARPS * 32), BAL_WARPS * 32, 0, st>>>(
      a, const_cast<SliceRec*>(rec), const_cast<unsigned long long*>(counts), const_cast<unsigned long long*>(woff),
      offsets, cap, keys, emit_gid);
  note_launch();
}

void launch_slice_emit_batch(const BatchItems& b, const SliceRec* rec, const unsigned long long* woff,
                             const unsigned long long* counts, unsigned long long* offsets, uint32_t cap,
                             uint32_t* keys, uint32_t* emit_gid, cudaStream_t st) {
  if (b.n_gauss <= 0) return;
  k_slice_bal_batch<true><<<ceil_div(b.n_gauss, BAL_WARPS * 32), BAL_WARPS * 32, 0, st>>>(
      b, const_cast<SliceRec*>(rec), const_cast<unsigned long long*>(counts), const_cast<unsigned long long*>(woff),
      offsets, cap, keys, emit_gid);
  note_launch();
}

// ------------------------------------------------------------ K-range
// Each thread takes RG_KEYS consecutive sorted keys (16-byte loads; the key
// array is 16-byte aligned and a vector that would run past the count is read
// key by key) and its neighbours' boundary keys by shuffle, so every key is
// loaded once.
constexpr int RG_KEYS = 16;

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ keys,
                                                const unsigned long long* __restrict__ n_dev, uint32_t cap,
                                                uint32_t nkeys, uint2* __restrict__ ranges) {
  const unsigned long long nn = *n_dev;
  const uint32_t n = nn < cap ? (uint32_t)nn : cap;
  const uint32_t i0 = (uint32_t)RG_KEYS * (blockIdx.x * blockDim.x + threadIdx.x);
  const int lane = threadIdx.x & 31;
  uint32_t k[RG_KEYS];
#pragma unroll
  for (int v = 0; v < RG_KEYS / 4; ++v) {
    const uint32_t j = i0 + 4u * (uint32_t)v;
    if (j + 4u <= n) {
      const uint4 q = *reinterpret_cast<const uint4*>(keys + j);
      k[4 * v] = q.x; k[4 * v + 1] = q.y; k[4 * v + 2] = q.z; k[4 * v + 3] = q.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) k[4 * v + q] = j + (uint32_t)q < n ? keys[j + q] : 0xffffffffu;
    }
  }
  uint32_t prev = __shfl_up_sync(0xffffffffu, k[RG_KEYS - 1], 1);
  uint32_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
  if (lane == 0) prev = (i0 > 0u && i0 - 1u < n) ? keys[i0 - 1u] : 0xffffffffu;
  if (lane == 31) next = i0 + (uint32_t)RG_KEYS < n ? keys[i0 + RG_KEYS] : 0xffffffffu;
#pragma unroll
  for (int j = 0; j < RG_KEYS; ++j) {
    const uint32_t i = i0 + (uint32_t)j;
    const uint32_t kj = k[j];
    if (i >= n) continue;
    if (kj >= nkeys) {  // cannot happen for emitted keys; keeps the store in bounds
      (void)GP_IN_RANGE(9, kj, nkeys);
      continue;
    }
    const uint32_t before = j == 0 ? prev : k[j - 1], after = j == RG_KEYS - 1 ? next : k[j + 1];
    if (i == 0u || before != kj) ranges[kj].x = i;
    if (i + 1u == n || after != kj) ranges[kj].y = i + 1u;
  }
}

void launch_ranges(const uint32_t* keys, const unsigned long long* n_dev, uint32_t cap, uint32_t nkeys,
                   uint2* ranges, cudaStream_t st) {
  if (cap == 0) return;
  const int64_t threads = ((int64_t)cap + RG_KEYS - 1) / RG_KEYS;
  k_ranges<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(keys, n_dev, cap, nkeys, ranges);
  note_launch();
}

// ------------------------------------------------------------ K-fwd
constexpr int FWD_CHUNK = 256;

// Per-(tile, slice) staging of one Gaussian: mu_2d relative to the tile origin
// (exact subtraction of the integer origin keeps pixel offsets accurate to a
// few 1e-7 px even 1000 px from the origin), a~, and the conic pre-scaled so
// that the exponent is already in base 2: e = c0 dx^2 + c1 dx dy + c2 dy^2.
//   s0 = (mu_2d,x - x0, mu_2d,y - y0, a~, C01),  s1 = (c0, c1, c2, C00)
template <int EXPM>
__device__ __forceinline__ void stage_gaussian(const SliceRec* __restrict__ rec, uint32_t g, float zsv,
                                               float x0, float y0, float4& s0, float4& s1, float& d,
                                               float& w, float& c11) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2);
  d = r0.z - zsv;
  w = exp2_sel<EXPM>(fmaxf(-0.5f * kLog2e * d * d * r0.w, kExpFloor));
  float mxr = (r0.x - x0) - r1.x * d;
  float myr = (r0.y - y0) - r1.y * d;
  s0 = make_float4(mxr, myr, r1.z * w, r2.y);
  s1 = make_float4(-0.5f * kLog2e * r2.x, -kLog2e * r2.y, -0.5f * kLog2e * r2.z, r2.x);
  c11 = r2.z;
}

// Per-thread forward of one (slice, tile) key of item a (local_key counts the
// item's own keys; ranges are batch-wide).
template <int TILE, int PX, int EXPM>
__device__ __forceinline__ void fwd_tile_px(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                            const uint32_t* __restrict__ vals, const uint32_t* __restrict__ emit_gid,
                                            const uint2* __restrict__ ranges, float* __restrict__ out) {
  constexpr int NT = TILE * TILE / PX;
  constexpr int SEGS = TILE / PX;
  __shared__ float4 s0[FWD_CHUNK], s1[FWD_CHUNK];
  const int T = a.TX * a.TY;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  const int row = threadIdx.x / SEGS, seg = threadIdx.x - row * SEGS;
  const float pyr = (float)row + 0.5f;
  const float px0 = (float)(seg * PX) + 0.5f;
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const float zsv = a.zorig[s];
  float acc[PX];
#pragma unroll
  for (int p = 0; p < PX; ++p) acc[p] = 0.0f;
  for (uint32_t base = rg.x; base < rg.y; base += FWD_CHUNK) {
    const int cnt = (int)min((uint32_t)FWD_CHUNK, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += NT) {
      const uint32_t v = vals[base + j];
      uint32_t g = emit_gid ? emit_gid[v] : v;
      float d, w, c11;
      float4 a0, a1;
      stage_gaussian<EXPM>(rec, g, zsv, x0, y0, a0, a1, d, w, c11);
      s0[j] = a0;
      s1[j] = a1;
    }
    __syncthreads();
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
      const float4 g0 = s0[j], g1 = s1[j];
      const float dy = pyr - g0.y;
      const float u = g1.y * dy;
      const float wy = g1.z * dy * dy;
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        float dx = (px0 + (float)p) - g0.x;
        float e = fmaf(dx, fmaf(g1.x, dx, u), wy);
        e = fmaxf(e, kExpFloor);
        acc[p] = fmaf(g0.z, exp2_sel<EXPM>(e), acc[p]);
      }
    }
    __syncthreads();
  }
  const int py = ty * TILE + row;
  if (py < a.H) {
    float* o = out + ((int64_t)s * a.H + py) * a.W + tx * TILE + seg * PX;
#pragma unroll
    for (int p = 0; p < PX; ++p)
      if (tx * TILE + seg * PX + p < a.W) o[p] = acc[p];
  }
}

template <int TILE, int PX, int EXPM>
__global__ void __launch_bounds__(TILE* TILE / PX) k_raster_fwd(SliceArgs a, const SliceRec* __restrict__ rec,
                                                               const uint32_t* __restrict__ vals,
                                                               const uint32_t* __restrict__ emit_gid,
                                                               const uint2* __restrict__ ranges,
                                                               float* __restrict__ out) {
  fwd_tile_px<TILE, PX, EXPM>(a, blockIdx.x, rec, vals, emit_gid, ranges, out);
}

template <int TILE, int PX, int EXPM>
__global__ void __launch_bounds__(TILE* TILE / PX) k_raster_fwd_px_batch(BatchItems b, const SliceRec* __restrict__ rec,
                                                                        const uint32_t* __restrict__ vals,
                                                                        const uint32_t* __restrict__ emit_gid,
                                                                        const uint2* __restrict__ ranges) {
  const uint32_t key = blockIdx.x;
  const int it = find_item_k(b.kstart, b.n_items, key);
  const SliceArgs a = b.args[it];
  if (a.out) fwd_tile_px<TILE, PX, EXPM>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, a.out);
}

template <int TILE, int PX>
static cudaError_t fwd_dispatch(const SliceArgs& a, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                                const uint32_t* emit_gid, const uint2* ranges, float* out, cudaStream_t st) {
  int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  if (tiles == 0) return cudaSuccess;
  constexpr int NT = TILE * TILE / PX;
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd<TILE, PX, GP_EXP_HW><<<(unsigned)tiles, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, out);
  else
    k_raster_fwd<TILE, PX, GP_EXP_POLY><<<(unsigned)tiles, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, out);
  note_launch();
  return cudaGetLastError();
}

template <int TILE, int PX>
static cudaError_t fwd_px_batch(const BatchItems& b, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                                const uint32_t* emit_gid, const uint2* ranges, cudaStream_t st) {
  constexpr int NT = TILE * TILE / PX;
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd_px_batch<TILE, PX, GP_EXP_HW><<<b.n_keys, NT, 0, st>>>(b, rec, vals, emit_gid, ranges);
  else
    k_raster_fwd_px_batch<TILE, PX, GP_EXP_POLY><<<b.n_keys, NT, 0, st>>>(b, rec, vals, emit_gid, ranges);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_raster_fwd_px_batch(const BatchItems& b, int tile, int px, int exp_mode, const SliceRec* rec,
                                       const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                       cudaStream_t st) {
  if (b.n_keys == 0) return cudaSuccess;
  if (exp_mode == GP_EXP_POLY_ROW) return cudaErrorInvalidValue;
  if (tile == 16 && px == 1) return fwd_px_batch<16, 1>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  if (tile == 16 && px == 2) return fwd_px_batch<16, 2>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  if (tile == 16 && px == 4) return fwd_px_batch<16, 4>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  if (tile == 8 && px == 1) return fwd_px_batch<8, 1>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  if (tile == 8 && px == 2) return fwd_px_batch<8, 2>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  return cudaErrorInvalidValue;
}

bool fwd_px_supported(int tile, int px) {
  return px == 0 || (tile == 16 ? (px == 1 || px == 2 || px == 4) : (tile == 8 ? (px == 1 || px == 2) : false));
}

cudaError_t launch_raster_fwd(const SliceArgs& a, int px, int raster, int exp_mode, const SliceRec* rec,
                              const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                              float* out, cudaStream_t st, uint32_t pairs) {
  if (px == 0) return launch_raster_fwd_blocked(a, raster, exp_mode, rec, vals, emit_gid, ranges, out, st, pairs);
  if (a.tile == 16) {
    switch (px) {
      case 1: return fwd_dispatch<16, 1>(a, exp_mode, rec, vals, emit_gid, ranges, out, st);
      case 2: return fwd_dispatch<16, 2>(a, exp_mode, rec, vals, emit_gid, ranges, out, st);
      case 4: return fwd_dispatch<16, 4>(a, exp_mode, rec, vals, emit_gid, ranges, out, st);
      default: return cudaErrorInvalidValue;
    }
  } else if (a.tile == 8) {
    switch (px) {
      case 1: return fwd_dispatch<8, 1>(a, exp_mode, rec, vals, emit_gid, ranges, out, st);
      case 2: return fwd_dispatch<8, 2>(a, exp_mode, rec, vals, emit_gid, ranges, out, st);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ K-bwd
// Accumulator layout, 10 floats per Gaussian (sums over its slices s):
//   0,1  S1 = sum dL/dmu_2d            2,3  S2 = sum delta dL/dmu_2d
//   4    T0 = sum dL/da~ w             5    T1 = sum dL/da~ w delta
//   6    T2 = sum dL/da~ w delta^2     7..9 sum dL/dC (C00, C01 as one symmetric
//                                           parameter, C11), C = Sigma_2d^-1
// with w = opacity_r of the slice.
constexpr int ACC = 10;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int TILE, int PX, int EXPM, bool DET>
__device__ __forceinline__ void bwd_tile_px(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                            const uint32_t* __restrict__ vals, const uint32_t* __restrict__ emit_gid,
                                            const uint2* __restrict__ ranges, const float* __restrict__ dL_dI,
                                            float* __restrict__ accum, float4* __restrict__ partial) {
  constexpr int NT = TILE * TILE / PX;
  constexpr int SEGS = TILE / PX;
  constexpr int NW = NT / 32;
  constexpr int CH = (NW >= 8) ? 64 : (NW >= 4 ? 128 : 256);
  __shared__ float4 s0[CH], s1[CH];
  __shared__ float4 s2[CH];            // (delta, w, C11, 0)
  __shared__ uint32_t sg[CH];          // Gaussian id
  __shared__ float sp[NW][6][CH];      // per-warp moments
  const int T = a.TX * a.TY;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  if (rg.y <= rg.x) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = threadIdx.x / SEGS, seg = threadIdx.x - row * SEGS;
  const float pyr = (float)row + 0.5f;
  const float px0 = (float)(seg * PX) + 0.5f;
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const float zsv = a.zorig[s];
  float G[PX];
  {
    const int py = ty * TILE + row;
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      const int px = tx * TILE + seg * PX + p;
      G[p] = (py < a.H && px < a.W) ? dL_dI[((int64_t)s * a.H + py) * a.W + px] : 0.0f;
    }
  }
  for (uint32_t base = rg.x; base < rg.y; base += CH) {
    const int cnt = (int)min((uint32_t)CH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += NT) {
      const uint32_t v = vals[base + j];
      uint32_t g = emit_gid ? emit_gid[v] : v;
      float d, w, c11;
      float4 a0, a1;
      stage_gaussian<EXPM>(rec, g, zsv, x0, y0, a0, a1, d, w, c11);
      s0[j] = a0;
      s1[j] = a1;
      s2[j] = make_float4(d, w, c11, 0.0f);
      sg[j] = g;
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float4 g0 = s0[j], g1 = s1[j];
      const float dy = pyr - g0.y;
      const float u = g1.y * dy;
      const float wy = g1.z * dy * dy;
      float m0 = 0.f, mx = 0.f, mxx = 0.f;
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        float dx = (px0 + (float)p) - g0.x;
        float e = fmaf(dx, fmaf(g1.x, dx, u), wy);
        e = fmaxf(e, kExpFloor);
        float gE = G[p] * exp2_sel_grad<EXPM>(e);
        m0 += gE;
        float tdx = gE * dx;
        mx += tdx;
        mxx = fmaf(tdx, dx, mxx);
      }
      // row moments -> the six moments of this lane
      float v0 = m0, v1 = mx, v2 = m0 * dy, v3 = mxx, v4 = mx * dy, v5 = v2 * dy;
      v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
      v3 = warp_sum(v3); v4 = warp_sum(v4); v5 = warp_sum(v5);
      if (lane == 0) {
        sp[warp][0][j] = v0; sp[warp][1][j] = v1; sp[warp][2][j] = v2;
        sp[warp][3][j] = v3; sp[warp][4][j] = v4; sp[warp][5][j] = v5;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += NT) {
      float m[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) acc += sp[w][k][j];
        m[k] = acc;
      }
      const float4 g0 = s0[j], g1 = s1[j];
      const float4 dw = s2[j];
      const float at = g0.z;  // a~
      const float C01 = g0.w, C00 = g1.w, C11 = dw.z;
      // pixel moments: m0 = sum G E, m1 = sum G E dx, m2 = sum G E dy,
      //                m3 = sum G E dx^2, m4 = sum G E dx dy, m5 = sum G E dy^2
      // dE/dmu_2d = E C d, dE/dC00 = -E dx^2 / 2, dE/dC01 = -E dx dy, dE/dC11 = -E dy^2 / 2
      const float g_at = m[0];
      const float gmx = at * (C00 * m[1] + C01 * m[2]);
      const float gmy = at * (C01 * m[1] + C11 * m[2]);
      const float gc00 = -0.5f * at * m[3];
      const float gc01 = -at * m[4];
      const float gc11 = -0.5f * at * m[5];
      if constexpr (DET) {
        uint32_t e = vals[base + j];
        partial[2 * (size_t)e] = make_float4(g_at, gmx, gmy, gc00);
        partial[2 * (size_t)e + 1] = make_float4(gc01, gc11, dw.x, dw.y);
      } else {
        float* A = accum + (size_t)sg[j] * ACC;
        const float d = dw.x, w = dw.y;
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

template <int TILE, int PX, int EXPM, bool DET>
__global__ void __launch_bounds__(TILE* TILE / PX) k_raster_bwd(
    SliceArgs a, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges,
    const float* __restrict__ dL_dI, float* __restrict__ accum, float4* __restrict__ partial) {
  bwd_tile_px<TILE, PX, EXPM, DET>(a, blockIdx.x, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
}

template <int TILE, int PX, int EXPM, bool DET>
__global__ void __launch_bounds__(TILE* TILE / PX) k_raster_bwd_px_batch(
    BatchItems b, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, float* __restrict__ accum,
    float4* __restrict__ partial) {
  const uint32_t key = blockIdx.x;
  const int it = find_item_k(b.kstart, b.n_items, key);
  const SliceArgs a = b.args[it];
  if (a.dL_dI)
    bwd_tile_px<TILE, PX, EXPM, DET>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, a.dL_dI, accum,
                                     partial);
}

template <int TILE, int PX>
static cudaError_t bwd_dispatch(const SliceArgs& a, int exp_mode, bool det, const SliceRec* rec,
                                const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                const float* dL_dI, float* accum, float4* partial, cudaStream_t st) {
  int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  if (tiles == 0) return cudaSuccess;
  constexpr int NT = TILE * TILE / PX;
  unsigned g = (unsigned)tiles;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd<TILE, PX, GP_EXP_HW, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
    else k_raster_bwd<TILE, PX, GP_EXP_HW, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
  } else {
    if (det) k_raster_bwd<TILE, PX, GP_EXP_POLY, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
    else k_raster_bwd<TILE, PX, GP_EXP_POLY, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, dL_dI, accum, partial);
  }
  note_launch();
  return cudaGetLastError();
}

template <int TILE, int PX>
static cudaError_t bwd_px_batch(const BatchItems& b, int exp_mode, bool det, const SliceRec* rec,
                                const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges, float* accum,
                                float4* partial, cudaStream_t st) {
  constexpr int NT = TILE * TILE / PX;
  const unsigned g = b.n_keys;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd_px_batch<TILE, PX, GP_EXP_HW, true><<<g, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_px_batch<TILE, PX, GP_EXP_HW, false><<<g, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial);
  } else {
    if (det) k_raster_bwd_px_batch<TILE, PX, GP_EXP_POLY, true><<<g, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_px_batch<TILE, PX, GP_EXP_POLY, false><<<g, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd_px_batch(const BatchItems& b, int tile, int px, int exp_mode, bool det,
                                       const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                       const uint2* ranges, float* accum, float4* partial, cudaStream_t st) {
  if (b.n_keys == 0) return cudaSuccess;
  if (exp_mode == GP_EXP_POLY_ROW) return cudaErrorInvalidValue;
  if (tile == 16 && px == 2) return bwd_px_batch<16, 2>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  if (tile == 16 && px == 4) return bwd_px_batch<16, 4>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  if (tile == 16 && px == 8) return bwd_px_batch<16, 8>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  if (tile == 8 && px == 2) return bwd_px_batch<8, 2>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  return cudaErrorInvalidValue;
}

bool bwd_px_supported(int tile, int px) {
  return px == 0 || (tile == 16 ? (px == 2 || px == 4 || px == 8) : (tile == 8 ? px == 2 : false));
}

cudaError_t launch_raster_bwd(const SliceArgs& a, int px, int raster, int exp_mode, bool det, const SliceRec* rec,
                              const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                              const float* dL_dI, float* accum, float4* partial, cudaStream_t st) {
  if (px == 0)
    return launch_raster_bwd_blocked(a, raster, exp_mode, det, rec, vals, emit_gid, ranges, dL_dI, accum, partial,
                                     st);
  if (a.tile == 16) {
    switch (px) {
      case 2: return bwd_dispatch<16, 2>(a, exp_mode, det, rec, vals, emit_gid, ranges, dL_dI, accum, partial, st);
      case 4: return bwd_dispatch<16, 4>(a, exp_mode, det, rec, vals, emit_gid, ranges, dL_dI, accum, partial, st);
      case 8: return bwd_dispatch<16, 8>(a, exp_mode, det, rec, vals, emit_gid, ranges, dL_dI, accum, partial, st);
      default: return cudaErrorInvalidValue;
    }
  } else if (a.tile == 8) {
    switch (px) {
      case 2: return bwd_dispatch<8, 2>(a, exp_mode, det, rec, vals, emit_gid, ranges, dL_dI, accum, partial, st);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ K-det
__global__ void k_det_reduce(int n, const unsigned long long* __restrict__ offsets,
                             const unsigned long long* __restrict__ counts,
                             const float4* __restrict__ partial, float* __restrict__ accum,
                             unsigned long long cap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float A[ACC];
#pragma unroll
  for (int k = 0; k < ACC; ++k) A[k] = 0.f;
  unsigned long long e0 = offsets[i], e1 = min(e0 + counts[i], cap);
  for (unsigned long long e = e0; e < e1; ++e) {
    float4 p0 = partial[2 * e], p1 = partial[2 * e + 1];
    const float g_at = p0.x, gmx = p0.y, gmy = p0.z, gc00 = p0.w, gc01 = p1.x, gc11 = p1.y;
    const float d = p1.z, w = p1.w, gw = g_at * w;
    A[0] += gmx; A[1] += gmy; A[2] += d * gmx; A[3] += d * gmy;
    A[4] += gw; A[5] += gw * d; A[6] += gw * d * d;
    A[7] += gc00; A[8] += gc01; A[9] += gc11;
  }
#pragma unroll
  for (int k = 0; k < ACC; ++k) accum[(size_t)i * ACC + k] = A[k];
}

void launch_det_reduce_n(int n, const unsigned long long* offsets, const unsigned long long* counts,
                         const float4* partial, float* accum, unsigned long long cap, cudaStream_t st) {
  if (n <= 0) return;
  k_det_reduce<<<ceil_div(n, 256), 256, 0, st>>>(n, offsets, counts, partial, accum, cap);
  note_launch();
}

// ------------------------------------------------------------ K-bwd-pre
// Closed-form chain from the ten accumulators to the parameters:
//   dL/dmu_p = S1,  dL/da = -S2,  dL/dmu_c = -a.S1 - A T1 / v,
//   dL/dA = T0 (dL/dalpha = T0 / sqrt(det)),  dL/ddet = -T0 A / (2 det),
//   dL/dv |_w = A T2 / (2 v^2),
//   dL/dSigma_2d = -C Gc C + dL/ddet det C   (Gc = symmetric dL/dC),
//   Sigma_2d = Sigma_pp - b b^T / v, a = b / v, v = Sigma_cc + sigma_z^2, b = Sigma_pc,
//   Sigma = M M^T, M = R diag(mod s), R = R(q/|q|).
// Gradients of Gaussian i of item a from the accumulators at batch-wide index ig.
__device__ __forceinline__ void slice_bwd_pre_one(const SliceArgs& a, int i, int ig, const float* __restrict__ accum,
                                                  float* __restrict__ d_mu, float* __restrict__ d_scale,
                                                  float* __restrict__ d_quat, float* __restrict__ d_alpha) {
  float acc[ACC];
#pragma unroll
  for (int k = 0; k < ACC; ++k) acc[k] = accum[(size_t)ig * ACC + k];
  float4 q = reinterpret_cast<const float4*>(a.quat)[i];
  float R[3][3], qn[4], qnorm;
  quat_rot(q, R, qn, qnorm);
  float dd[3] = {a.mod * a.scale[3 * i], a.mod * a.scale[3 * i + 1], a.mod * a.scale[3 * i + 2]};
  float M[3][3], Sw[6];
  covariance(R, dd, M, Sw);
  float mc[3], Sc[6];
  camera_frame(a.Rc, a.tc, a.mu + 3 * i, Sw, mc, Sc);
  float cxx = Sc[0], cxy = Sc[1], cxz = Sc[2], cyy = Sc[3], cyz = Sc[4], czz = Sc[5];
  float v = czz + a.sigma2, iv = 1.0f / v;
  float ax = cxz * iv, ay = cyz * iv;
  float sxx = cxx - cxz * ax, sxy = cxy - cxz * ay, syy = cyy - cyz * ay;
  float det = sxx * syy - sxy * sxy;
  bool valid = det > 1e-30f && isfinite(det) && qnorm > 0.0f;
  float gmu[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, galpha = 0.f;
  if (valid) {
    float idet = 1.0f / det, sq = sqrtf(det);
    // amplitude A = alpha / sqrt(det) (slices) or alpha (voxelizer planes, no det term)
    float A = a.vox ? a.alpha[i] : a.alpha[i] / sq;
    float C00 = syy * idet, C01 = -sxy * idet, C11 = sxx * idet;
    const float S1x = acc[0], S1y = acc[1], S2x = acc[2], S2y = acc[3];
    const float T0 = acc[4], T1 = acc[5], T2 = acc[6];
    const float G00 = acc[7], G01 = 0.5f * acc[8], G11 = acc[9];
    galpha = a.vox ? T0 : T0 / sq;
    float gdet = a.vox ? 0.0f : -0.5f * T0 * A * idet;
    // dL/dSigma_2d = -C Gc C + gdet det C  (symmetric)
    float CG00 = C00 * G00 + C01 * G01, CG01 = C00 * G01 + C01 * G11;
    float CG10 = C01 * G00 + C11 * G01, CG11 = C01 * G01 + C11 * G11;
    float H00 = -(CG00 * C00 + CG01 * C01) + gdet * det * C00;
    float H01 = -(CG00 * C01 + CG01 * C11) + gdet * det * C01;
    float H11 = -(CG10 * C01 + CG11 * C11) + gdet * det * C11;
    float gax = -S2x, gay = -S2y;
    float Hbx = H00 * cxz + H01 * cyz, Hby = H01 * cxz + H11 * cyz;
    float gv = A * T2 * iv * iv * 0.5f + (cxz * Hbx + cyz * Hby) * iv * iv - (gax * cxz + gay * cyz) * iv * iv;
    float gbx = -2.0f * Hbx * iv + gax * iv, gby = -2.0f * Hby * iv + gay * iv;
    float gmc[3] = {S1x, S1y, -(ax * S1x + ay * S1y) - A * iv * T1};
    // camera frame -> world: dL/dmu = R_c^T dL/dmu_c, dL/dSigma = R_c^T dL/dSigma_c R_c
    const float* Rc = a.Rc;
    float Gc[3][3] = {{H00, H01, 0.5f * gbx}, {H01, H11, 0.5f * gby}, {0.5f * gbx, 0.5f * gby, gv}};
    float GR[3][3];  // Gc R_c
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        GR[u][l] = fmaf(Gc[u][2], Rc[6 + l], fmaf(Gc[u][1], Rc[3 + l], Gc[u][0] * Rc[l]));
    float Gw[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gmu[k] = fmaf(Rc[6 + k], gmc[2], fmaf(Rc[3 + k], gmc[1], Rc[k] * gmc[0]));
#pragma unroll
      for (int l = 0; l < 3; ++l)
        Gw[k][l] = fmaf(Rc[6 + k], GR[2][l], fmaf(Rc[3 + k], GR[1][l], Rc[k] * GR[0][l]));
    }
    scale_quat_backward(R, M, dd, qn, qnorm, a.mod, Gw, gs, gq);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d_mu[3 * i + k] = gmu[k];
    d_scale[3 * i + k] = gs[k];
  }
  reinterpret_cast<float4*>(d_quat)[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
  d_alpha[i] = galpha;
}

__global__ void __launch_bounds__(PRE_THREADS) k_slice_bwd_pre(SliceArgs a, const float* __restrict__ accum,
                                                               float* __restrict__ d_mu,
                                                               float* __restrict__ d_scale,
                                                               float* __restrict__ d_quat,
                                                               float* __restrict__ d_alpha) {
  const int i = blockIdx.x * PRE_THREADS + threadIdx.x;
  if (i < a.n) slice_bwd_pre_one(a, i, i, accum, d_mu, d_scale, d_quat, d_alpha);
}

__global__ void __launch_bounds__(PRE_THREADS) k_slice_bwd_pre_batch(BatchItems b, const float* __restrict__ accum) {
  const int ig = blockIdx.x * PRE_THREADS + threadIdx.x;
  if (ig >= b.n_gauss) return;
  const int k = find_item(b.gstart, b.n_items, ig);
  const SliceArgs a = b.args[k];
  if (!a.d_mu) return;  // item without gradient outputs
  slice_bwd_pre_one(a, ig - b.gstart[k], ig, accum, a.d_mu, a.d_scale, a.d_quat, a.d_alpha);
}

void launch_slice_bwd_pre_batch(const BatchItems& b, const float* accum, cudaStream_t st) {
  if (b.n_gauss <= 0) return;
  k_slice_bwd_pre_batch<<<ceil_div(b.n_gauss, PRE_THREADS), PRE_THREADS, 0, st>>>(b, accum);
  note_launch();
}

void launch_slice_bwd_pre(const SliceArgs& a, const float* accum, float* d_mu, float* d_scale,
                          float* d_quat, float* d_alpha, cudaStream_t st) {
  if (a.n <= 0) return;
  k_slice_bwd_pre<<<ceil_div(a.n, PRE_THREADS), PRE_THREADS, 0, st>>>(a, accum, d_mu, d_scale, d_quat,
                                                                      d_alpha);
  note_launch();
}

// ------------------------------------------------------------ K-loss
constexpr int MSE_THREADS = 256;
constexpr int MSE_ITEMS = 8;

__global__ void __launch_bounds__(MSE_THREADS) k_mse(const float* __restrict__ I, const float* __restrict__ T,
                                                     const int* __restrict__ t_index, int64_t HW, int bpsl,
                                                     float scale, float* __restrict__ g,
                                                     float* __restrict__ part) {
  __shared__ float sw[MSE_THREADS / 32];
  const int s = blockIdx.x / bpsl, b = blockIdx.x - s * bpsl;
  const int64_t ts = t_index ? (int64_t)t_index[s] : (int64_t)s;
  const float* Is = I + (int64_t)s * HW;
  const float* Ts = T + ts * HW;
  float* gs = g + (int64_t)s * HW;
  float acc = 0.f;
  for (int64_t i = (int64_t)b * MSE_THREADS + threadIdx.x; i < HW; i += (int64_t)bpsl * MSE_THREADS) {
    float r = Is[i] - Ts[i];
    gs[i] = 2.0f * r * scale;
    acc = fmaf(r, r, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < MSE_THREADS / 32; ++w) t += sw[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_mse_final(const float* __restrict__ part, int nb, float scale, float* __restrict__ loss) {
  __shared__ float sw[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sw[w];
    *loss = t * scale;
  }
}

static int mse_blocks_per_slice(int64_t HW) {
  int64_t b = (HW + (int64_t)MSE_THREADS * MSE_ITEMS - 1) / ((int64_t)MSE_THREADS * MSE_ITEMS);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

int mse_tmp_floats(int S, int64_t HW) { return S * mse_blocks_per_slice(HW); }

void launch_mse(const float* I, const float* T, const int* t_index, int S, int64_t HW, float* dL_dI,
                float* loss, float* tmp, cudaStream_t st) {
  if (S <= 0 || HW <= 0) return;
  int bpsl = mse_blocks_per_slice(HW);
  float scale = 1.0f / ((float)S * (float)HW);
  k_mse<<<S * bpsl, MSE_THREADS, 0, st>>>(I, T, t_index, HW, bpsl, scale, dL_dI, tmp);
  note_launch();
  if (loss) {
    k_mse_final<<<1, 1024, 0, st>>>(tmp, S * bpsl, scale, loss);
    note_launch();
  }
}

// ------------------------------------------------------------ counting
// Pixels of one (Gaussian, slice, tile) inside d^T C d <= k2: per row, the
// interval of dx solving the quadratic, intersected with the tile.
__global__ void __launch_bounds__(PRE_THREADS) k_count_evals(SliceArgs a, const SliceRec* __restrict__ rec,
                                                             unsigned long long* __restrict__ out) {
  int i = blockIdx.x * PRE_THREADS + threadIdx.x;
  unsigned long long cnt = 0;
  if (i < a.n) {
    SliceRec r = rec[i];
    const float c00 = r.r2.x, c01 = r.r2.y, c11 = r.r2.z;
    for_each_pair(a, r, [&](int j, int tile) {
      float d = r.r0.z - a.zs[j];
      float mx = r.r0.x - r.r1.x * d, my = r.r0.y - r.r1.y * d;
      int ty = tile / a.TX, tx = tile - ty * a.TX;
      int xa = tx * a.tile, xb = min((tx + 1) * a.tile, a.W);
      if (a.vox) {
        // voxelizer plane: the section of the 3D ellipsoid, d^T C d <= k2 - delta^2 / Sigma_zz,
        // in double precision (the count is compared with an FP64 lattice count)
        const double dd = (double)r.r0.z - (double)a.zs[j];
        const double k2e = (double)a.k2 - dd * dd * (double)r.r0.w;
        const double mxd = (double)r.r0.x - (double)r.r1.x * dd, myd = (double)r.r0.y - (double)r.r1.y * dd;
        for (int y = ty * a.tile; y < min((ty + 1) * a.tile, a.H); ++y) {
          const double dy = (double)y + 0.5 - myd;
          const double disc = (double)c01 * c01 * dy * dy - (double)c00 * ((double)c11 * dy * dy - k2e);
          if (!(disc >= 0.0)) continue;
          const double sq = sqrt(disc);
          const double lo = mxd + (-(double)c01 * dy - sq) / c00, hi = mxd + (-(double)c01 * dy + sq) / c00;
          int x0 = max(xa, (int)ceil(lo - 0.5)), x1 = min(xb - 1, (int)floor(hi - 0.5));
          if (x1 >= x0) cnt += (unsigned long long)(x1 - x0 + 1);
        }
        return;
      }
      for (int y = ty * a.tile; y < min((ty + 1) * a.tile, a.H); ++y) {
        float dy = (float)y + 0.5f - my;
        float disc = c01 * c01 * dy * dy - c00 * (c11 * dy * dy - a.k2);
        if (disc < 0.f) continue;
        float sq = sqrtf(disc);
        float lo = mx + (-c01 * dy - sq) / c00, hi = mx + (-c01 * dy + sq) / c00;
        // pixels x with x + 0.5 in [lo, hi]
        int x0 = max(xa, (int)ceilf(lo - 0.5f)), x1 = min(xb - 1, (int)floorf(hi - 0.5f));
        if (x1 >= x0) cnt += (unsigned long long)(x1 - x0 + 1);
      }
    });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

void launch_count_evals(const SliceArgs& a, const SliceRec* rec, unsigned long long* out, cudaStream_t st) {
  if (a.n <= 0) return;
  k_count_evals<<<ceil_div(a.n, PRE_THREADS), PRE_THREADS, 0, st>>>(a, rec, out);
  note_launch();
}

// Pixels the default rasterisers evaluate, out[0] forward and out[1]
// backward: row units (rows): 8 per (Gaussian, plane, tile, column band,
// pixel row) whose segment of pixel centres the culling ellipse meets;
// block-culled: 64 per 8 x 8 block (forward) and 32 per 8 x 4 half-block
// (backward) the ellipse touches -- the same tests the kernels stage with.
template <int TILE>
__global__ void __launch_bounds__(PRE_THREADS) k_count_units(SliceArgs a, const SliceRec* __restrict__ rec,
                                                             bool rows_f, bool rows_b,
                                                             unsigned long long* __restrict__ out) {
  int i = blockIdx.x * PRE_THREADS + threadIdx.x;
  unsigned long long cnt = 0, cntb = 0;
  if (i < a.n) {
    const SliceRec r = rec[i];
    for_each_pair(a, r, [&](int j, int tile) {
      const int ty = tile / a.TX, tx = tile - ty * a.TX;
      const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
      const float d = r.r0.z - a.zs[j];
      const float mx = (r.r0.x - x0) - r.r1.x * d, my = (r.r0.y - y0) - r.r1.y * d;
      const int nrows = min(TILE, a.H - ty * TILE), nbands = min(TILE / 8, (a.W - tx * TILE + 7) >> 3);
      const unsigned long long units =
          (rows_f || rows_b)
              ? 8ull * (unsigned)__popc(row_unit_mask<TILE>(r.r0, r.r2, r.r3, d, mx, my, a.k2, a.vox != 0, nrows,
                                                             nbands))
              : 0ull;
      cnt += rows_f ? units : 64ull * (unsigned)__popc(plane_cells<TILE, 8>(r.r0, r.r2, r.r3, d, mx, my, a.k2,
                                                                            a.vox != 0));
      cntb += rows_b ? units : 32ull * (unsigned)__popc(plane_cells<TILE, 4>(r.r0, r.r2, r.r3, d, mx, my, a.k2,
                                                                             a.vox != 0));
    });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    cntb += __shfl_xor_sync(0xffffffffu, cntb, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
  if ((threadIdx.x & 31) == 0 && cntb) atomicAdd(out + 1, cntb);
}

void launch_count_units(const SliceArgs& a, const SliceRec* rec, bool rows_f, bool rows_b, unsigned long long* out,
                        cudaStream_t st) {
  if (a.tile == 8)
    k_count_units<8><<<ceil_div(a.n, PRE_THREADS), PRE_THREADS, 0, st>>>(a, rec, rows_f, rows_b, out);
  else
    k_count_units<16><<<ceil_div(a.n, PRE_THREADS), PRE_THREADS, 0, st>>>(a, rec, rows_f, rows_b, out);
  note_launch();
}

__global__ void k_exp2_eval(const float* __restrict__ x, float* __restrict__ y, int64_t n, int mode) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = fmaxf(x[i], kExpFloor);
  if (mode == GP_EXP_POLY_PACKED || mode == GP_EXP_POLY_GRAD_PACKED) {
    // the packed two-value form, paired with the neighbouring element
    const int64_t j = i ^ 1;
    const float w = j < n ? fmaxf(x[j], kExpFloor) : 0.0f;
    const float2 xv = (i & 1) ? make_float2(w, v) : make_float2(v, w);
    const float2 r = mode == GP_EXP_POLY_PACKED ? exp2_poly2(xv) : exp2_grad2(xv);
    y[i] = (i & 1) ? r.y : r.x;
    return;
  }
  y[i] = mode == GP_EXP_HW ? exp2_hw(v) : mode == GP_EXP_POLY_GRAD ? exp2_grad(v) : exp2_poly(v);
}

void launch_exp2_eval(const float* x, float* y, int64_t n, int mode, cudaStream_t st) {
  if (n <= 0) return;
  k_exp2_eval<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n, mode);
  note_launch();
}

GP_CHECK_READER(check_read_slice)

}  // namespace gp
