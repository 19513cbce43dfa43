// raster.cu -- block-culled tile rasterisers of the slice renderer (the default
// K-fwd and K-bwd), sm_103a; plain (one CTA per tile) and persistent (a work
// queue over every tile of a batch of renders) launches share the tile bodies.
//
// A CTA owns one (slice, tile) and its binned Gaussian list.  Gaussians are
// staged in shared memory in chunks (16-byte loads of the 64-byte records, mu_2d
// and a~ of this slice computed once per Gaussian), and at staging each one's
// culling ellipse d^T Sigma_2d^-1 d <= k^2 (k^2 = 2 ln(1/eps)) is turned into a
// mask of the tile's cells it touches, from its x-extent over each band of
// pixel rows.
//
// Forward: the warps own the 8x8 blocks of the tile (four for 16x16 tiles, one
// for 8x8).  Per chunk each warp compacts the staged Gaussians whose mask has
// its block; its four 8-lane groups take four of them at a time, lane r of a
// group evaluating row r of the block (8 pixels): along a row the exponent is a
// quadratic in the pixel offset q from the block's centre column, two pixels
// per packed fp32x2 instruction.  Each lane keeps 8 partial sums per group; the
// four groups are added in a fixed shuffle tree at the end, so results are
// bitwise reproducible.
// Backward: after the tile's dL/dI is in shared memory every warp works on its
// own chunks of the list without block barriers.  The unit of work is a
// (Gaussian, 8x4 half-block) pair the mask marks; one lane evaluates a unit's
// 32 pixels and forms its six moments sum G E {1, dx, dy, dx^2, dx dy, dy^2}
// (E the Gaussian's exponential, G = dL/dI).  The unit list is Gaussian-major,
// so a segmented scan over the lanes sums each Gaussian's units into its six
// accumulators in a fixed order; the accumulators are then folded into the 10
// per-Gaussian sums (atomics) or written as a per-pair partial (deterministic
// mode).
// GP_EXP_POLY_ROW factors the exponential along each row (two exp2 per 8
// pixels, see row_powers) in both kernels.
// The sorted list values are Gaussian ids (emit_gid == nullptr) or, in the
// deterministic mode, emission indices mapped through emit_gid.  The forward is
// built twice, for 8 CTAs per SM on dense tiles (more registers, more
// exponentials in flight) and 12 on sparse ones; the launcher picks by the
// mean number of pairs per tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "gp_check.cuh"
#include "gp_common.cuh"
#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

// Staging of one Gaussian for one (slice, tile):
//   s0 = (mu_2d,x - x0, mu_2d,y - y0, a~, C11)
//   s1 = (c0, c1, c2, C00)     e = c0 dx^2 + c1 dx dy + c2 dy^2 = -log2(e)/2 d^T C d
//   s2 = (delta, opacity_r, C01, 0)    (backward)
// and the mask of the cells (bands of BH rows) its culling ellipse touches.
// On a voxelizer plane (vox) the culling ellipse is the plane's section of the
// 3D one, d^T C d <= k2 - delta^2 / Sigma_zz (its extents scaled to match).
template <int EXPM, int TILE, int BH>
__device__ __forceinline__ unsigned stage_blk(const SliceRec* __restrict__ rec, uint32_t g, float zsv, float x0,
                                              float y0, float k2, bool vox, float4& s0, float4& s1, float4& s2) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2), r3 = __ldg(rp + 3);
  const float d = r0.z - zsv;
  const float w = exp2_sel<EXPM>(fmaxf(-0.5f * kLog2e * d * d * r0.w, kExpFloor));
  const float mxr = (r0.x - x0) - r1.x * d;
  const float myr = (r0.y - y0) - r1.y * d;
  const float C00 = r2.x, C01 = r2.y, C11 = r2.z;
  s0 = make_float4(mxr, myr, r1.z * w, C11);
  s1 = make_float4(-0.5f * kLog2e * C00, -kLog2e * C01, -0.5f * kLog2e * C11, C00);
  s2 = make_float4(d, w, C01, 0.0f);
  return plane_cells<TILE, BH>(r0, r2, r3, d, mxr, myr, k2, vox);
}

// ---- row factorisation (GP_EXP_POLY_ROW)
// Along a row the exponent is e(q) = A + B q + C q^2 (C < 0), q = p - 3.5 for
// the pixels p = 0..7.  With j the pixel's distance in pixels from the row's end
// where the linear part A + B q is larger (j = 7 - p if B >= 0, j = p if not),
//     2^e(q) = 2^(A + 3.5 |B|) * (2^-|B|)^j * 2^(C q^2),
// i.e. two exp2 per row (L = 2^(A + 3.5|B|), r = 2^-|B|), powers of r by
// multiplication and four per-Gaussian values 2^(C q^2), q^2 in {1/4, 9/4,
// 25/4, 49/4}.  Every factor but L is <= 1, and since e(q) <= 0 for all real q,
// A + 3.5 |B| <= 12.25 |C|: with |C| <= 8 L stays below 2^98 and 2^(C q^2)
// above 2^-98, so no factor overflows and a factor underflows only where the
// product is below 2^-51.  Narrower Gaussians (C < kRowMinC, a conditional
// standard deviation under 0.3 pixel) take the per-pixel exp2.
constexpr float kRowMinC = -8.0f;

template <int EXPM>
constexpr bool row_factored() { return EXPM == GP_EXP_POLY_ROW; }

// 2^(c q^2) for q = 3.5, 2.5, 1.5, 0.5 (fa) and 0.5, 1.5, 2.5, 3.5 (fb), times s.
__device__ __forceinline__ void row_quad_factors(float c, float s, float4& fa, float4& fb) {
  const float2 e01 = exp2_poly2(make_float2(fmaxf(0.25f * c, kExpFloor), fmaxf(2.25f * c, kExpFloor)));
  const float2 e23 = exp2_poly2(make_float2(fmaxf(6.25f * c, kExpFloor), fmaxf(12.25f * c, kExpFloor)));
  const float2 s01 = __fmul2_rn(e01, make_float2(s, s)), s23 = __fmul2_rn(e23, make_float2(s, s));
  fa = make_float4(s23.y, s23.x, s01.y, s01.x);
  fb = make_float4(s01.x, s01.y, s23.x, s23.y);
}

// L and r^0..r^7 of one row, as the pairs (r^0, r^1) ... (r^6, r^7) scaled by
// L (forward) or not (backward, which applies L to the row's sums).
struct RowPowers {
  float L;
  float2 p01, p23, p45, p67;
};

__device__ __forceinline__ RowPowers row_powers(float A, float aB, bool scale_by_L) {
  const float2 ex = exp2_poly2(make_float2(fmaxf(fmaf(3.5f, aB, A), kExpFloor), fmaxf(-aB, kExpFloor)));
  const float r = ex.y, r2 = r * r;
  const float2 r23 = make_float2(r2, r2 * r);
  const float2 r45 = __fmul2_rn(make_float2(r2, r2), r23);          // r^4, r^5
  const float2 r67 = __fmul2_rn(make_float2(r45.x, r45.x), r23);    // r^6, r^7
  RowPowers w;
  w.L = ex.x;
  if (scale_by_L) {
    const float2 L2 = make_float2(ex.x, ex.x);
    w.p01 = make_float2(ex.x, ex.x * r);
    w.p23 = __fmul2_rn(L2, r23);
    w.p45 = __fmul2_rn(L2, r45);
    w.p67 = __fmul2_rn(L2, r67);
  } else {
    w.p01 = make_float2(1.0f, r);
    w.p23 = r23;
    w.p45 = r45;
    w.p67 = r67;
  }
  return w;
}

// The backward's powers of one row in mirrored couples: L, (r^0, r^1),
// (r^2, r^3) for the distances 0..3 from the row's larger end, and (r^7, r^6),
// (r^5, r^4) for their mirrors 7..4.
struct RowCouplePowers {
  float L;
  float2 p01, p23, p76, p54;
};

__device__ __forceinline__ RowCouplePowers row_couple_powers(float A, float aB) {
  const float2 ex = exp2_poly2(make_float2(fmaxf(fmaf(3.5f, aB, A), kExpFloor), fmaxf(-aB, kExpFloor)));
  const float r = ex.y, r2 = r * r, r3 = r2 * r, r4 = r2 * r2;
  const float2 r32 = make_float2(r3, r2);
  RowCouplePowers w;
  w.L = ex.x;
  w.p01 = make_float2(1.0f, r);
  w.p23 = make_float2(r2, r3);
  w.p54 = __fmul2_rn(make_float2(r2, r2), r32);
  w.p76 = __fmul2_rn(make_float2(r4, r4), r32);
  return w;
}

// Shared memory of the forward body.
template <int TILE, int CH, bool RF = false>
struct FwdSmem {
  float4 s0[CH], s1[CH];
  float4 fa[RF ? CH : 1], fb[RF ? CH : 1];   // row factorisation: a~ 2^(C q^2) per pixel column
  unsigned char bmask[CH];                   // per Gaussian: the 8 x 8 blocks its ellipse touches
  int hitlist[(TILE / 8) * (TILE / 8)][CH];  // per warp: the chunk's Gaussians that hit its block
};

// One (slice s, tile t) of item a: every pixel of the tile is written.
template <int TILE, int CH, int EXPM>
__device__ __forceinline__ void fwd_tile(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                         const uint32_t* __restrict__ vals, const uint32_t* __restrict__ emit_gid,
                                         const uint2* __restrict__ ranges,
                                         FwdSmem<TILE, CH, row_factored<EXPM>()>& sm) {
  constexpr int NT = (TILE / 8) * (TILE / 8) * 32;
  constexpr bool RF = row_factored<EXPM>();
  const int T = a.TX * a.TY;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  if (!GP_IN_RANGE(6, local_key, T * a.S)) return;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> 3, row = lane & 7;
  const float bx = (float)((warp % (TILE / 8)) * 8), by = (float)((warp / (TILE / 8)) * 8);
  const float pyr = by + (float)row + 0.5f;
  const float cxb = bx + 4.0f;  // centre column of the block's 8 pixel centres
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const float zsv = a.zorig[s];
  int* list = sm.hitlist[warp];
  float2 acc[4];  // pixels (2p, 2p + 1) of the lane's row
#pragma unroll
  for (int p = 0; p < 4; ++p) acc[p] = make_float2(0.0f, 0.0f);
  for (uint32_t base = rg.x; base < rg.y; base += CH) {
    const int cnt = (int)min((uint32_t)CH, rg.y - base);
    for (int j = threadIdx.x; j < cnt; j += NT) {
      float4 a0, a1, a2;
      const uint32_t v = vals[base + j];
      const uint32_t g = emit_gid ? emit_gid[v] : v;  // sorted values: emission indices, or Gaussian ids
      sm.bmask[j] = GP_IN_RANGE(5, (int64_t)g - a.gbase, a.n)
                        ? (unsigned char)stage_blk<EXPM, TILE, 8>(rec, g, zsv, x0, y0, a.k2, a.vox != 0, a0, a1, a2)
                        : (unsigned char)0;
      sm.s0[j] = a0;
      sm.s1[j] = a1;
      if constexpr (RF) {
        float4 fa, fb;
        row_quad_factors(a1.x, a0.z, fa, fb);
        sm.fa[j] = fa;
        sm.fb[j] = fb;
      }
    }
    __syncthreads();
    // test the whole chunk first, so that the hits are taken four at a time
    // with at most one partly idle round per chunk
    int nh = 0;
    for (int jb = 0; jb < cnt; jb += 32) {
      const int j = jb + lane;
      const bool hit = j < cnt && ((sm.bmask[j] >> warp) & 1u);
      const unsigned msk = __ballot_sync(0xffffffffu, hit);
      const int at = nh + __popc(msk & ((1u << lane) - 1u));
      if (hit && GP_IN_RANGE(4, at, CH)) list[at] = j;
      nh += __popc(msk);
    }
    __syncwarp();
    {
      for (int h = grp; h < nh; h += 4) {
        const int jj = list[h];
        const float4 g0 = sm.s0[jj], g1 = sm.s1[jj];
        // along the row, with q = p - 3.5 the pixel offset from the block's centre
        // column, the exponent is A + B q + C q^2
        const float dy = pyr - g0.y;
        const float u = g1.y * dy;
        const float dxc = cxb - g0.x;
        const float A = fmaf(dxc, fmaf(g1.x, dxc, u), g1.z * dy * dy);
        const float Bq = fmaf(2.0f * g1.x, dxc, u);
        if (RF && g1.x >= kRowMinC) {
          // pixel p takes L r^j a~ 2^(C q^2), j = 7 - p when B >= 0 and p otherwise
          const RowPowers w = row_powers(A, fabsf(Bq), true);
          const bool rev = Bq >= 0.0f;
          const float4 fa = sm.fa[jj], fb = sm.fb[jj];
          const float2 W0 = rev ? make_float2(w.p67.y, w.p67.x) : w.p01;
          const float2 W1 = rev ? make_float2(w.p45.y, w.p45.x) : w.p23;
          const float2 W2 = rev ? make_float2(w.p23.y, w.p23.x) : w.p45;
          const float2 W3 = rev ? make_float2(w.p01.y, w.p01.x) : w.p67;
          acc[0] = __ffma2_rn(W0, make_float2(fa.x, fa.y), acc[0]);
          acc[1] = __ffma2_rn(W1, make_float2(fa.z, fa.w), acc[1]);
          acc[2] = __ffma2_rn(W2, make_float2(fb.x, fb.y), acc[2]);
          acc[3] = __ffma2_rn(W3, make_float2(fb.z, fb.w), acc[3]);
        } else {
          const float2 C2 = make_float2(g1.x, g1.x), B2 = make_float2(Bq, Bq), A2 = make_float2(A, A);
          const float2 at2 = make_float2(g0.z, g0.z);
          // two pixels per packed instruction; each lane of a pair is rounded as
          // the scalar form would round it
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float2 q = make_float2((float)(2 * p) - 3.5f, (float)(2 * p + 1) - 3.5f);
            acc[p] = __ffma2_rn(at2, pair_exp2<EXPM>(C2, B2, A2, q), acc[p]);
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // the four groups' partial sums of the same pixels, in a fixed tree
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    acc[p].x += __shfl_xor_sync(0xffffffffu, acc[p].x, 8);
    acc[p].y += __shfl_xor_sync(0xffffffffu, acc[p].y, 8);
    acc[p].x += __shfl_xor_sync(0xffffffffu, acc[p].x, 16);
    acc[p].y += __shfl_xor_sync(0xffffffffu, acc[p].y, 16);
  }
  if (grp == 0) {
    const int py = ty * TILE + (int)by + row;
    const int px0 = tx * TILE + (int)bx;
    if (py < a.H) {
      float* o = a.out + ((int64_t)s * a.H + py) * a.W + px0;
      if (px0 + 8 <= a.W && ((((uintptr_t)o) & 15u) == 0)) {
        reinterpret_cast<float4*>(o)[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
        reinterpret_cast<float4*>(o)[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
      } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (px0 + 2 * p < a.W) o[2 * p] = acc[p].x;
          if (px0 + 2 * p + 1 < a.W) o[2 * p + 1] = acc[p].y;
        }
      }
    }
  }
}

constexpr int ACC10 = 10;

// Shared memory of the backward body.  The tile's dL/dI is held half-block by
// half-block (4 rows of 8 pixels each), the half-blocks 36 floats apart: the
// 16-byte loads of the same row and column by lanes working on different
// half-blocks then fall in different banks.  A row is stored as its pixels
// 0, 1, 2, 3, 7, 6, 5, 4 (each pixel of the first half followed, four places on,
// by its mirror about the row's centre), or in order with a reversed copy
// beside it under the row factorisation.
template <int TILE, int CH, bool RF = false>
struct BwdSmem {
  static constexpr int NW = (TILE / 8) * (TILE / 8);
  static constexpr int NH = 2 * NW;  // 8 x 4 half-blocks per tile
  static constexpr int HBS = 36;     // floats per half-block (32 + 4 of padding)
  float4 s0[CH], s1[CH], s2[CH];
  float4 fa[RF ? CH : 1];  // row factorisation: 2^(C q^2), |q| = 3.5, 2.5, 1.5, 0.5
  uint32_t sg[CH];
  alignas(16) float G[NH * HBS];
  alignas(16) float Grev[RF ? NH * HBS : 4];  // row factorisation: G with each row of 8 reversed
  int units[NW][CH * NH / NW];  // per warp: the hit (Gaussian, half-block) pairs it tested, (j << 4) | hb
  float acc[6][CH];             // per Gaussian: the six pixel moments summed over its half-blocks
};

// Backward of one (slice s, tile t) of item a.  The tile is cut into 8 x 4
// half-blocks; every (staged Gaussian, half-block) pair whose ellipse touches
// the half-block is a unit of work.  Each warp takes its own chunks of the
// tile's list and evaluates their units one per lane: a lane sums, over its
// unit's 32 pixels, the six moments
//     sum G E {1, dx, dy, dx^2, dx dy, dy^2}      (E the Gaussian's exponential,
// G = dL/dI, d = pixel - mu_2d), row by row with two pixels per packed
// instruction and a row's pixels in mirrored couples.  The per-half-block
// moments of a Gaussian are summed in a fixed order and folded into its 10
// accumulators (atomics) or written as a per-pair partial (deterministic
// mode).
template <int TILE, int CH, int EXPM, bool DET>
__device__ __forceinline__ void bwd_tile(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                         const uint32_t* __restrict__ vals, const uint32_t* __restrict__ emit_gid,
                                         const uint2* __restrict__ ranges, float* __restrict__ accum,
                                         float4* __restrict__ partial,
                                         BwdSmem<TILE, CH, row_factored<EXPM>()>& sm) {
  constexpr bool RF = row_factored<EXPM>();
  constexpr int NW = BwdSmem<TILE, CH, RF>::NW;
  constexpr int NH = BwdSmem<TILE, CH, RF>::NH;
  constexpr int HBS = BwdSmem<TILE, CH, RF>::HBS;
  constexpr int NT = NW * 32;
  constexpr int CW = CH / NW;  // Gaussians per warp chunk
  static_assert(CW * NH == CH * NH / NW && CW * NH % 32 == 0 && NH <= 8 && (NH & (NH - 1)) == 0,
                "tile / chunk shape");
  const int T = a.TX * a.TY;
  if (!GP_IN_RANGE(6, local_key, T * a.S)) return;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  if (rg.y <= rg.x) return;  // uniform over the CTA
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const float zsv = a.zorig[s];
  // the tile's dL/dI (zero outside the image), half-block-major
  for (int i = threadIdx.x; i < TILE * TILE; i += NT) {
    const int yy = i / TILE, xx = i - yy * TILE;
    const int py = ty * TILE + yy, px = tx * TILE + xx;
    const int hb = 2 * ((yy >> 3) * (TILE / 8) + (xx >> 3)) + ((yy >> 2) & 1);
    const float gv = (py < a.H && px < a.W) ? a.dL_dI[((int64_t)s * a.H + py) * a.W + px] : 0.0f;
    const int cx = xx & 7;
    sm.G[hb * HBS + (yy & 3) * 8 + ((RF || cx < 4) ? cx : 11 - cx)] = gv;
    if constexpr (RF) sm.Grev[hb * HBS + (yy & 3) * 8 + (7 - (xx & 7))] = gv;
  }
  __syncthreads();
  // From here on every warp works alone on its own chunks of the list: it
  // stages CW Gaussians into its own slots with the half-blocks each one's
  // ellipse touches, evaluates those units and folds them, so a Gaussian's
  // units never leave the warp and warps need no block-wide barrier.
  const int slot0 = warp * CW;
  int* units = sm.units[warp];
  for (uint32_t base = rg.x + (uint32_t)slot0; base < rg.y; base += CH) {
    const int cnt = (int)min((uint32_t)CW, rg.y - base);
    // stage the chunk and list its (Gaussian, half-block) units, Gaussian-major
    // with half-blocks ascending: a warp scan of the units per Gaussian gives
    // each lane where to write its own
    int nu = 0;
    for (int jl0 = 0; jl0 < cnt; jl0 += 32) {
      const int jl = jl0 + lane;
      const int j = slot0 + jl;
      unsigned hm = 0u;
      if (jl < cnt) {
        const uint32_t v = vals[base + jl];
        const uint32_t g = emit_gid ? emit_gid[v] : v;  // sorted values: emission indices, or Gaussian ids
        float4 a0, a1, a2;
        if (GP_IN_RANGE(5, (int64_t)g - a.gbase, a.n))
          hm = stage_blk<EXPM, TILE, 4>(rec, g, zsv, x0, y0, a.k2, a.vox != 0, a0, a1, a2);
        sm.s0[j] = a0;
        sm.s1[j] = a1;
        sm.s2[j] = a2;
        sm.sg[j] = g;
#pragma unroll
        for (int k = 0; k < 6; ++k) sm.acc[k][j] = 0.0f;
        if constexpr (RF) {
          float4 fa, fb;
          row_quad_factors(a1.x, 1.0f, fa, fb);
          sm.fa[j] = fa;  // the couples use 2^(C q^2) in the order |q| = 3.5, 2.5, 1.5, 0.5 only
        }
      }
      const int c = __popc(hm);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int sh = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += sh;
      }
      int at = nu + incl - c;
      while (hm) {
        const int hb = __ffs(hm) - 1;
        hm &= hm - 1u;
        if (GP_IN_RANGE(1, at, CW * NH)) units[at] = (j << 4) | hb;
        ++at;
      }
      nu += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // units in rounds of 32; the units of one Gaussian are consecutive (the
    // list is Gaussian-major), so after each round a segmented scan over the
    // lanes sums them and the segment's last lane adds the sum to the
    // Gaussian's accumulators (a fixed order: the sums are reproducible)
    for (int u0 = 0; u0 < nu; u0 += 32) {
      const int u = u0 + lane;
      const bool valid = u < nu;
      const int code = valid ? units[u] : -16;  // an idle lane is its own segment, Gaussian -1
      const int jj = code >> 4, hb = code & 15;
      const bool ok = valid && GP_IN_RANGE(2, jj - slot0, CW) && GP_IN_RANGE(3, hb, NH);
      float mom[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (ok) {
        const float4 g0 = sm.s0[jj], g1 = sm.s1[jj];
        const float c0 = g1.x, c1 = g1.y, c2 = g1.z;
        const int hbx = ((hb >> 1) % (TILE / 8)) * 8, hby = ((hb >> 1) / (TILE / 8)) * 8 + 4 * (hb & 1);
        const float dxc = (float)hbx + 4.0f - g0.x, dy0 = (float)hby + 0.5f - g0.y;
        // row r of the half-block: exponent A(r) + B(r) q + c0 q^2 along the row,
        // q the offset from the half-block's centre column
        const float A0 = fmaf(dxc, fmaf(c0, dxc, c1 * dy0), c2 * dy0 * dy0);
        const float A1 = fmaf(c1, dxc, 2.0f * c2 * dy0);
        const float B0 = fmaf(2.0f * c0, dxc, c1 * dy0);
        const float2 C2 = make_float2(c0, c0);
        float M00 = 0.f, M10 = 0.f, M20 = 0.f, M01 = 0.f, M11 = 0.f, M02 = 0.f;
        const float* Gr = sm.G + hb * HBS;
        if (RF && c0 >= kRowMinC) {
          // rows in the factored form, over j (the distance from the row's
          // larger end), in mirrored couples (j, 7 - j): the pixel of j has
          // q = j - 3.5 when B < 0 and 3.5 - j when B >= 0, so in that frame a
          // couple is (q, -q) as in the per-pixel form below.  The near half
          // (j = 0..3) comes from the tile's dL/dI in the row's order, the far
          // half (j = 7..4) from the reversed copy, or the other way round.
          const float4 fa = sm.fa[jj];
          const float2 F0 = make_float2(fa.x, fa.y), F1 = make_float2(fa.z, fa.w);  // 2^(C q^2), |q| = 3.5, 2.5 / 1.5, 0.5
          const float* Grv = sm.Grev + hb * HBS;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float rf = (float)r;
            const float A = fmaf(fmaf(c2, rf, A1), rf, A0);
            const float B = fmaf(c1, rf, B0);
            const RowCouplePowers w = row_couple_powers(A, fabsf(B));
            const bool rev = B >= 0.0f;
            const float4 gn = *reinterpret_cast<const float4*>((rev ? Grv : Gr) + r * 8);  // j = 0, 1, 2, 3
            const float4 gf = *reinterpret_cast<const float4*>((rev ? Gr : Grv) + r * 8);  // j = 7, 6, 5, 4
            // sum G E = X + Y, sum q G E = q (X + Y) - 2 q Y, sum q^2 G E = q^2 (X + Y)
            // couple 0: j = (0, 1) with (7, 6), q = (-3.5, -2.5)
            float2 P0, P1, P2;
            {
              const float2 Y = __fmul2_rn(make_float2(gf.x, gf.y), __fmul2_rn(w.p76, F0));
              const float2 XY = __ffma2_rn(make_float2(gn.x, gn.y), __fmul2_rn(w.p01, F0), Y);
              P0 = XY;
              P1 = __ffma2_rn(make_float2(7.0f, 5.0f), Y, __fmul2_rn(make_float2(-3.5f, -2.5f), XY));
              P2 = __fmul2_rn(make_float2(12.25f, 6.25f), XY);
            }
            // couple 1: j = (2, 3) with (5, 4), q = (-1.5, -0.5)
            {
              const float2 Y = __fmul2_rn(make_float2(gf.z, gf.w), __fmul2_rn(w.p54, F1));
              const float2 XY = __ffma2_rn(make_float2(gn.z, gn.w), __fmul2_rn(w.p23, F1), Y);
              P0 = __fadd2_rn(P0, XY);
              P1 = __ffma2_rn(make_float2(3.0f, 1.0f), Y, __ffma2_rn(make_float2(-1.5f, -0.5f), XY, P1));
              P2 = __ffma2_rn(make_float2(2.25f, 0.25f), XY, P2);
            }
            const float S0 = w.L * (P0.x + P0.y);
            const float S1 = (rev ? -w.L : w.L) * (P1.x + P1.y);
            const float S2 = w.L * (P2.x + P2.y);
            M00 += S0;
            M10 += S1;
            M20 += S2;
            M01 = fmaf(rf, S0, M01);
            M11 = fmaf(rf, S1, M11);
            M02 = fmaf(rf * rf, S0, M02);
          }
        } else {
          // per-pixel exponentials, the pixels of a row taken in mirrored couples
          // (q, -q): with X = G E at the q < 0 pixels and Y at their mirrors,
          //     sum G E = X + Y,  sum q G E = q (X + Y) - 2 q Y,  sum q^2 G E = q^2 (X + Y).
          // Rows run bottom-up with running sums P, so the row-weighted moments
          // are sums of P's snapshots: sum_r r S_r = s3 + (s3 + s2) + (s3 + s2 + s1)
          // and sum_r r^2 S_r = 5 s3 + 3 (s3 + s2) + (s3 + s2 + s1) (s_r the row sums).
          const float* Gm = RF ? sm.Grev + hb * HBS : Gr + 4;  // the row's pixels 7, 6, 5, 4
          // the exponent is concave in (q, r): if its four corners are above
          // kExpUnfloored, so is every pixel, and the pixels need no floor
          const float Bl = fmaf(c1, 3.0f, B0), Al = fmaf(fmaf(c2, 3.0f, A1), 3.0f, A0);
          const float emin = fminf(fmaf(-3.5f, fabsf(B0), fmaf(12.25f, c0, A0)),
                                   fmaf(-3.5f, fabsf(Bl), fmaf(12.25f, c0, Al)));
          auto rows = [&](auto floor_tag) {
            constexpr bool FL = decltype(floor_tag)::value;
            float2 P0, P1, P2, T0, T1, U0;
  #pragma unroll
            for (int r = 3; r >= 0; --r) {
              const float rf = (float)r;
              const float A = fmaf(fmaf(c2, rf, A1), rf, A0);
              const float B = fmaf(c1, rf, B0);
              const float2 A2 = make_float2(A, A), B2 = make_float2(B, B), Bn2 = make_float2(-B, -B);
              const float4 gx = *reinterpret_cast<const float4*>(Gr + r * 8);
              const float4 gy = *reinterpret_cast<const float4*>(Gm + r * 8);
  #pragma unroll
              for (int k = 0; k < 2; ++k) {
                const float qa = (float)(2 * k) - 3.5f, qb = qa + 1.0f;
                const float2 q = make_float2(qa, qb), q2 = make_float2(qa * qa, qb * qb);
                const float2 GX = k == 0 ? make_float2(gx.x, gx.y) : make_float2(gx.z, gx.w);
                const float2 GY = k == 0 ? make_float2(gy.x, gy.y) : make_float2(gy.z, gy.w);
                // e(+-q) = (A + C q^2) +- B q
                const float2 base = __ffma2_rn(C2, q2, A2);
                const float2 Y = __fmul2_rn(GY, couple_exp2<EXPM, FL, true>(Bn2, q, base));
                const float2 XY = __ffma2_rn(GX, couple_exp2<EXPM, FL, true>(B2, q, base), Y);
                if (r == 3 && k == 0) {
                  P0 = XY;
                  P1 = __fmul2_rn(q, XY);
                  P2 = __fmul2_rn(q2, XY);
                } else {
                  P0 = __fadd2_rn(P0, XY);
                  P1 = __ffma2_rn(q, XY, P1);
                  P2 = __ffma2_rn(q2, XY, P2);
                }
                P1 = __ffma2_rn(make_float2(-2.0f * qa, -2.0f * qb), Y, P1);
              }
              if (r == 3) {
                T0 = P0;
                T1 = P1;
                U0 = __fmul2_rn(make_float2(5.0f, 5.0f), P0);
              } else if (r == 2) {
                T0 = __fadd2_rn(T0, P0);
                T1 = __fadd2_rn(T1, P1);
                U0 = __ffma2_rn(make_float2(3.0f, 3.0f), P0, U0);
              } else if (r == 1) {
                T0 = __fadd2_rn(T0, P0);
                T1 = __fadd2_rn(T1, P1);
                U0 = __fadd2_rn(U0, P0);
              }
            }
            M00 = P0.x + P0.y;
            M10 = P1.x + P1.y;
            M20 = P2.x + P2.y;
            M01 = T0.x + T0.y;
            M11 = T1.x + T1.y;
            M02 = U0.x + U0.y;
          };
          if (__all_sync(__activemask(), emin >= kExpUnfloored))
            rows(std::false_type{});
          else
            rows(std::true_type{});
        }
        // moments in d = (dxc + q, dy0 + r)
        mom[0] = M00;
        mom[1] = fmaf(dxc, M00, M10);
        mom[2] = fmaf(dy0, M00, M01);
        mom[3] = fmaf(dxc, fmaf(dxc, M00, 2.0f * M10), M20);
        mom[4] = fmaf(dxc, fmaf(dy0, M00, M01), fmaf(dy0, M10, M11));
        mom[5] = fmaf(dy0, fmaf(dy0, M00, 2.0f * M01), M02);
      }
      // segmented inclusive scan: a Gaussian has at most NH units, so offsets
      // 1, 2, ..., NH / 2 reach the whole segment
      const int jprev = __shfl_up_sync(0xffffffffu, jj, 1);
      const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || jprev != jj);
      const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
      for (int o = 1; o < NH; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float t = __shfl_up_sync(0xffffffffu, mom[k], o);
          if (lane - o >= start) mom[k] += t;
        }
      }
      const int jnext = __shfl_down_sync(0xffffffffu, jj, 1);
      if (ok && (lane == 31 || u + 1 == nu || jnext != jj)) {
#pragma unroll
        for (int k = 0; k < 6; ++k) sm.acc[k][jj] += mom[k];
      }
    }
    __syncwarp();
    for (int jl = lane; jl < cnt; jl += 32) {
      const int j = slot0 + jl;
      float m[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) m[k] = sm.acc[k][j];
      const float4 g0 = sm.s0[j], g1 = sm.s1[j], g2 = sm.s2[j];
      const float at = g0.z;
      const float C00 = g1.w, C01 = g2.z, C11 = g0.w;
      // dE/dmu_2d = E C d; dE/dC00 = -E dx^2/2, dE/dC01 = -E dx dy, dE/dC11 = -E dy^2/2
      const float g_at = m[0];
      const float gmx = at * (C00 * m[1] + C01 * m[2]);
      const float gmy = at * (C01 * m[1] + C11 * m[2]);
      const float gc00 = -0.5f * at * m[3];
      const float gc01 = -at * m[4];
      const float gc11 = -0.5f * at * m[5];
      const float d = g2.x, w = g2.y;
      if constexpr (DET) {
        const uint32_t e = vals[base + jl];
        partial[2 * (size_t)e] = make_float4(g_at, gmx, gmy, gc00);
        partial[2 * (size_t)e + 1] = make_float4(gc01, gc11, d, w);
      } else {
        float* A = accum + (size_t)sm.sg[j] * ACC10;
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
    __syncwarp();
  }
}

}  // namespace gp

#include "raster_rows.cuh"

namespace gp {

// ------------------------------------------------------------ plain kernels
// Row-unit kernels (the default for per-pixel exponentials): one warp per tile.
// The forward runs one warp per CTA (69 registers, 24 CTAs per SM: fewer
// registers for more resident warps slowed it, 1.01 -> 1.05 ms at 63 and 1.09 ms
// at 48).  The backward runs two tiles per CTA, each warp with its own shared
// memory and no barrier between them: 62 registers and 32 resident warps per SM
// (one warp per CTA reached fewer, limited by the CTAs an SM holds; voxelizer
// planes' backward 1.44 -> 1.25 ms).
constexpr int kRowCtasPerSm = 24;
constexpr int kRowBwdWarps = 2, kRowBwdCtasPerSm = 16;

template <int TILE, int EXPM>
__global__ void __launch_bounds__(32, kRowCtasPerSm) k_raster_fwd_rows(SliceArgs a, const SliceRec* __restrict__ rec,
                                                                       const uint32_t* __restrict__ vals,
                                                                       const uint32_t* __restrict__ emit_gid,
                                                                       const uint2* __restrict__ ranges) {
  if constexpr (TILE == 16) {
    __shared__ OwnFwdSmem sm;
    fwd_tile_owner<EXPM>(a, blockIdx.x, rec, vals, emit_gid, ranges, sm);
  } else {
    __shared__ RowFwdSmem<TILE> sm;
    fwd_tile_rows<TILE, EXPM>(a, blockIdx.x, rec, vals, emit_gid, ranges, sm);
  }
}

template <int TILE, int EXPM, bool DET>
__global__ void __launch_bounds__(32 * kRowBwdWarps, kRowBwdCtasPerSm) k_raster_bwd_rows(
    SliceArgs a, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, float* __restrict__ accum,
    float4* __restrict__ partial) {
  const int w = threadIdx.x >> 5, key = blockIdx.x * kRowBwdWarps + w;
  if ((int64_t)key >= (int64_t)a.S * a.TX * a.TY) return;  // the last CTA's spare warp
  __shared__ RowBwdSmem<TILE> sm[kRowBwdWarps];
  bwd_tile_rows<TILE, EXPM, DET>(a, key, rec, vals, emit_gid, ranges, accum, partial, sm[w]);
}

// Block-culled kernels (the row-factored exponential's): four warps per 16 x 16 tile.
template <int TILE, int CH, int EXPM, bool DENSE>
__global__ void __launch_bounds__((TILE / 8) * (TILE / 8) * 32, TILE == 16 ? (DENSE ? 8 : 12) : 32) k_raster_fwd_blk(
    SliceArgs a, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges) {
  __shared__ FwdSmem<TILE, CH, row_factored<EXPM>()> sm;
  fwd_tile<TILE, CH, EXPM>(a, blockIdx.x, rec, vals, emit_gid, ranges, sm);
}

template <int TILE, int CH, int EXPM, bool DET>
__global__ void __launch_bounds__((TILE / 8) * (TILE / 8) * 32, TILE == 16 ? 9 : 32)
    k_raster_bwd_blk(SliceArgs a, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
                     const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges,
                     float* __restrict__ accum, float4* __restrict__ partial) {
  __shared__ BwdSmem<TILE, CH, row_factored<EXPM>()> sm;
  bwd_tile<TILE, CH, EXPM, DET>(a, blockIdx.x, rec, vals, emit_gid, ranges, accum, partial, sm);
}

// ------------------------------------------------------- persistent kernels
// Every CTA takes chunks of KEY_CHUNK consecutive keys from the work counter and
// renders each (item, slice, tile) key of the chunk; the item of a key is found
// by binary search over the items' key starts.
constexpr int KEY_CHUNK = 8;


template <int TILE, int CH, int EXPM>
__global__ void __launch_bounds__((TILE / 8) * (TILE / 8) * 32, TILE == 16 ? 12 : 32) k_raster_fwd_persist(
    BatchItems b, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, unsigned* __restrict__ work) {
  __shared__ FwdSmem<TILE, CH, row_factored<EXPM>()> sm;
  __shared__ uint32_t next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(work, (unsigned)KEY_CHUNK);
    __syncthreads();
    const uint32_t k0 = next;
    __syncthreads();
    if (k0 >= b.n_keys) break;
    const uint32_t k1 = min(k0 + (uint32_t)KEY_CHUNK, b.n_keys);
    for (uint32_t key = k0; key < k1; ++key) {
      const int it = find_item_k(b.kstart, b.n_items, key);
      const SliceArgs a = b.args[it];
      if (a.out) fwd_tile<TILE, CH, EXPM>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, sm);
      __syncthreads();
    }
  }
}

template <int TILE, int CH, int EXPM, bool DET>
__global__ void __launch_bounds__((TILE / 8) * (TILE / 8) * 32, TILE == 16 ? (row_factored<EXPM>() ? 9 : 10) : 32)
    k_raster_bwd_persist(
    BatchItems b, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, float* __restrict__ accum,
    float4* __restrict__ partial, unsigned* __restrict__ work) {
  __shared__ BwdSmem<TILE, CH, row_factored<EXPM>()> sm;
  __shared__ uint32_t next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(work, (unsigned)KEY_CHUNK);
    __syncthreads();
    const uint32_t k0 = next;
    __syncthreads();
    if (k0 >= b.n_keys) break;
    const uint32_t k1 = min(k0 + (uint32_t)KEY_CHUNK, b.n_keys);
    for (uint32_t key = k0; key < k1; ++key) {
      const int it = find_item_k(b.kstart, b.n_items, key);
      const SliceArgs a = b.args[it];
      if (a.dL_dI) bwd_tile<TILE, CH, EXPM, DET>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, accum,
                                                 partial, sm);
      __syncthreads();
    }
  }
}

// Persistent row-unit kernels: each warp takes chunks of keys.
template <int TILE, int EXPM>
__global__ void __launch_bounds__(32, kRowCtasPerSm) k_raster_fwd_rows_persist(
    BatchItems b, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, unsigned* __restrict__ work) {
  using Smem = typename std::conditional<TILE == 16, OwnFwdSmem, RowFwdSmem<TILE>>::type;
  __shared__ Smem sm;
  for (;;) {
    uint32_t k0 = 0;
    if (threadIdx.x == 0) k0 = atomicAdd(work, (unsigned)KEY_CHUNK);
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    if (k0 >= b.n_keys) break;
    const uint32_t k1 = min(k0 + (uint32_t)KEY_CHUNK, b.n_keys);
    for (uint32_t key = k0; key < k1; ++key) {
      const int it = find_item_k(b.kstart, b.n_items, key);
      const SliceArgs a = b.args[it];
      if (a.out) {
        if constexpr (TILE == 16)
          fwd_tile_owner<EXPM>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, sm);
        else
          fwd_tile_rows<TILE, EXPM>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, sm);
      }
      __syncwarp();
    }
  }
}

// The backward's CTAs hold kRowBwdWarps warps, each taking its own chunks.
template <int TILE, int EXPM, bool DET>
__global__ void __launch_bounds__(32 * kRowBwdWarps, kRowBwdCtasPerSm) k_raster_bwd_rows_persist(
    BatchItems b, const SliceRec* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ emit_gid, const uint2* __restrict__ ranges, float* __restrict__ accum,
    float4* __restrict__ partial, unsigned* __restrict__ work) {
  __shared__ RowBwdSmem<TILE> smw[kRowBwdWarps];
  RowBwdSmem<TILE>& sm = smw[threadIdx.x >> 5];
  for (;;) {
    uint32_t k0 = 0;
    if ((threadIdx.x & 31) == 0) k0 = atomicAdd(work, (unsigned)KEY_CHUNK);
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    if (k0 >= b.n_keys) break;
    const uint32_t k1 = min(k0 + (uint32_t)KEY_CHUNK, b.n_keys);
    for (uint32_t key = k0; key < k1; ++key) {
      const int it = find_item_k(b.kstart, b.n_items, key);
      const SliceArgs a = b.args[it];
      if (a.dL_dI) bwd_tile_rows<TILE, EXPM, DET>(a, (int)(key - b.kstart[it]), rec, vals, emit_gid, ranges, accum,
                                                  partial, sm);
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------ launchers
template <int TILE>
static cudaError_t fwd_rows(const SliceArgs& a, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                            const uint32_t* emit_gid, const uint2* ranges, cudaStream_t st) {
  const unsigned tiles = (unsigned)((int64_t)a.S * a.TX * a.TY);
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd_rows<TILE, GP_EXP_HW><<<tiles, 32, 0, st>>>(a, rec, vals, emit_gid, ranges);
  else
    k_raster_fwd_rows<TILE, GP_EXP_POLY><<<tiles, 32, 0, st>>>(a, rec, vals, emit_gid, ranges);
  note_launch();
  return cudaGetLastError();
}

template <int TILE>
static cudaError_t bwd_rows(const SliceArgs& a, int exp_mode, bool det, const SliceRec* rec, const uint32_t* vals,
                            const uint32_t* emit_gid, const uint2* ranges, float* accum, float4* partial,
                            cudaStream_t st) {
  const unsigned tiles = (unsigned)((int64_t)a.S * a.TX * a.TY);
  const unsigned g = (tiles + kRowBwdWarps - 1) / kRowBwdWarps;
  constexpr int NT = 32 * kRowBwdWarps;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd_rows<TILE, GP_EXP_HW, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_rows<TILE, GP_EXP_HW, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
  } else {
    if (det) k_raster_bwd_rows<TILE, GP_EXP_POLY, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_rows<TILE, GP_EXP_POLY, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
  }
  note_launch();
  return cudaGetLastError();
}

template <int TILE, int CH, bool DENSE>
static cudaError_t fwd_blk(const SliceArgs& a, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                           const uint32_t* emit_gid, const uint2* ranges, cudaStream_t st) {
  const int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  constexpr int NT = (TILE / 8) * (TILE / 8) * 32;
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd_blk<TILE, CH, GP_EXP_HW, DENSE><<<(unsigned)tiles, NT, 0, st>>>(a, rec, vals, emit_gid, ranges);
  else if (exp_mode == GP_EXP_POLY_ROW)
    k_raster_fwd_blk<TILE, CH, GP_EXP_POLY_ROW, DENSE><<<(unsigned)tiles, NT, 0, st>>>(a, rec, vals, emit_gid, ranges);
  else
    k_raster_fwd_blk<TILE, CH, GP_EXP_POLY, DENSE><<<(unsigned)tiles, NT, 0, st>>>(a, rec, vals, emit_gid, ranges);
  note_launch();
  return cudaGetLastError();
}

bool raster_rows_form(const SliceArgs& a, int raster, int exp_mode, bool backward) {
  if (exp_mode == GP_EXP_POLY_ROW) return false;
  return raster == GP_RASTER_ROWS || (raster == GP_RASTER_AUTO && (!backward || a.vox != 0));
}

cudaError_t launch_raster_fwd_blocked(const SliceArgs& a, int raster, int exp_mode, const SliceRec* rec,
                                      const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges, float* out,
                                      cudaStream_t st, uint32_t pairs) {
  const int64_t tiles = (int64_t)a.S * a.TX * a.TY;
  if (tiles == 0) return cudaSuccess;
  SliceArgs b = a;
  b.out = out;
  if (raster_rows_form(a, raster, exp_mode, false)) {
    if (a.tile == 16) return fwd_rows<16>(b, exp_mode, rec, vals, emit_gid, ranges, st);
    if (a.tile == 8) return fwd_rows<8>(b, exp_mode, rec, vals, emit_gid, ranges, st);
    return cudaErrorInvalidValue;
  }
  if (a.tile == 16) {
    if ((int64_t)pairs >= (int64_t)kDenseTilePairs * tiles)
      return fwd_blk<16, 128, true>(b, exp_mode, rec, vals, emit_gid, ranges, st);
    return fwd_blk<16, 128, false>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  }
  if (a.tile == 8) return fwd_blk<8, 64, false>(b, exp_mode, rec, vals, emit_gid, ranges, st);
  return cudaErrorInvalidValue;
}

template <int TILE, int CH>
static cudaError_t bwd_blk(const SliceArgs& a, int exp_mode, bool det, const SliceRec* rec, const uint32_t* vals,
                           const uint32_t* emit_gid, const uint2* ranges, float* accum, float4* partial,
                           cudaStream_t st) {
  const unsigned g = (unsigned)((int64_t)a.S * a.TX * a.TY);
  constexpr int NT = (TILE / 8) * (TILE / 8) * 32;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd_blk<TILE, CH, GP_EXP_HW, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_blk<TILE, CH, GP_EXP_HW, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
  } else if (exp_mode == GP_EXP_POLY_ROW) {
    if (det) k_raster_bwd_blk<TILE, CH, GP_EXP_POLY_ROW, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_blk<TILE, CH, GP_EXP_POLY_ROW, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
  } else {
    if (det) k_raster_bwd_blk<TILE, CH, GP_EXP_POLY, true><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
    else k_raster_bwd_blk<TILE, CH, GP_EXP_POLY, false><<<g, NT, 0, st>>>(a, rec, vals, emit_gid, ranges, accum, partial);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd_blocked(const SliceArgs& a, int raster, int exp_mode, bool det, const SliceRec* rec,
                                      const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                      const float* dL_dI, float* accum, float4* partial, cudaStream_t st) {
  if ((int64_t)a.S * a.TX * a.TY == 0) return cudaSuccess;
  SliceArgs b = a;
  b.dL_dI = dL_dI;
  if (raster_rows_form(a, raster, exp_mode, true)) {
    if (a.tile == 16) return bwd_rows<16>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
    if (a.tile == 8) return bwd_rows<8>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
    return cudaErrorInvalidValue;
  }
  if (a.tile == 16) return bwd_blk<16, 128>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  if (a.tile == 8) return bwd_blk<8, 32>(b, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, st);
  return cudaErrorInvalidValue;
}

// Persistent launchers: chunk in {64, 128, 256} Gaussians per staging round.
template <int TILE, int CH>
static cudaError_t fwd_persist(const BatchItems& b, int ctas, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                               const uint32_t* emit_gid, const uint2* ranges, unsigned* work, cudaStream_t st) {
  constexpr int NT = (TILE / 8) * (TILE / 8) * 32;
  if (exp_mode == GP_EXP_HW)
    k_raster_fwd_persist<TILE, CH, GP_EXP_HW><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, work);
  else if (exp_mode == GP_EXP_POLY_ROW)
    k_raster_fwd_persist<TILE, CH, GP_EXP_POLY_ROW><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, work);
  else
    k_raster_fwd_persist<TILE, CH, GP_EXP_POLY><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, work);
  note_launch();
  return cudaGetLastError();
}

template <int TILE, int CH>
static cudaError_t bwd_persist(const BatchItems& b, int ctas, int exp_mode, bool det, const SliceRec* rec,
                               const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges, float* accum,
                               float4* partial, unsigned* work, cudaStream_t st) {
  constexpr int NT = (TILE / 8) * (TILE / 8) * 32;
  if (exp_mode == GP_EXP_HW) {
    if (det) k_raster_bwd_persist<TILE, CH, GP_EXP_HW, true><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
    else k_raster_bwd_persist<TILE, CH, GP_EXP_HW, false><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
  } else if (exp_mode == GP_EXP_POLY_ROW) {
    if (det) k_raster_bwd_persist<TILE, CH, GP_EXP_POLY_ROW, true><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
    else k_raster_bwd_persist<TILE, CH, GP_EXP_POLY_ROW, false><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
  } else {
    if (det) k_raster_bwd_persist<TILE, CH, GP_EXP_POLY, true><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
    else k_raster_bwd_persist<TILE, CH, GP_EXP_POLY, false><<<ctas, NT, 0, st>>>(b, rec, vals, emit_gid, ranges, accum, partial, work);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_raster_fwd_batch(const BatchItems& b, bool rows, int tile, int chunk, int ctas, int exp_mode,
                                    const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                    const uint2* ranges, unsigned* work, cudaStream_t st) {
  if (b.n_keys == 0) return cudaSuccess;
  if (rows && exp_mode != GP_EXP_POLY_ROW) {
#define GP_FWD_R(T, E) \
  if (tile == T && exp_mode == E) {                                                              \
    k_raster_fwd_rows_persist<T, E><<<ctas, 32, 0, st>>>(b, rec, vals, emit_gid, ranges, work);  \
    note_launch();                                                                               \
    return cudaGetLastError();                                                                   \
  }
    GP_FWD_R(16, GP_EXP_POLY) GP_FWD_R(16, GP_EXP_HW) GP_FWD_R(8, GP_EXP_POLY) GP_FWD_R(8, GP_EXP_HW)
#undef GP_FWD_R
    return cudaErrorInvalidValue;
  }
#define GP_FWD_P(T, C) \
  if (tile == T && chunk == C) return fwd_persist<T, C>(b, ctas, exp_mode, rec, vals, emit_gid, ranges, work, st);
  GP_FWD_P(16, 64) GP_FWD_P(16, 128) GP_FWD_P(16, 256) GP_FWD_P(8, 64) GP_FWD_P(8, 128) GP_FWD_P(8, 256)
#undef GP_FWD_P
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_bwd_batch(const BatchItems& b, bool rows, int tile, int chunk, int ctas, int exp_mode, bool det,
                                    const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                    const uint2* ranges, float* accum, float4* partial, unsigned* work,
                                    cudaStream_t st) {
  if (b.n_keys == 0) return cudaSuccess;
  if (rows && exp_mode != GP_EXP_POLY_ROW) {
#define GP_BWD_R(T, E)                                                                                         \
  if (tile == T && exp_mode == E) {                                                                            \
    if (det)                                                                                                   \
      k_raster_bwd_rows_persist<T, E, true><<<ctas, 32 * kRowBwdWarps, 0, st>>>(b, rec, vals, emit_gid, ranges,  \
                                                                                accum, partial, work);           \
    else                                                                                                       \
      k_raster_bwd_rows_persist<T, E, false><<<ctas, 32 * kRowBwdWarps, 0, st>>>(b, rec, vals, emit_gid, ranges, \
                                                                                 accum, partial, work);          \
    note_launch();                                                                                             \
    return cudaGetLastError();                                                                                 \
  }
    GP_BWD_R(16, GP_EXP_POLY) GP_BWD_R(16, GP_EXP_HW) GP_BWD_R(8, GP_EXP_POLY) GP_BWD_R(8, GP_EXP_HW)
#undef GP_BWD_R
    return cudaErrorInvalidValue;
  }
#define GP_BWD_P(T, C)                                                                                       \
  if (tile == T && chunk == C)                                                                               \
    return bwd_persist<T, C>(b, ctas, exp_mode, det, rec, vals, emit_gid, ranges, accum, partial, work, st);
  GP_BWD_P(16, 32) GP_BWD_P(16, 64) GP_BWD_P(16, 128) GP_BWD_P(8, 32) GP_BWD_P(8, 64) GP_BWD_P(8, 128)
#undef GP_BWD_P
  return cudaErrorInvalidValue;
}

// Resident CTAs per SM of a persistent kernel (occupancy calculator).
int raster_batch_ctas_per_sm(bool rows, int tile, int chunk, bool backward, int exp_mode) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const bool row = exp_mode == GP_EXP_POLY_ROW;
  if (rows && !row) {  // the row-unit kernels (warps of their own; the chunk is fixed at 32 Gaussians)
    constexpr int NB = 32 * kRowBwdWarps;
    if (tile == 16)
      e = backward ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_bwd_rows_persist<16, GP_EXP_POLY, false>, NB, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd_rows_persist<16, GP_EXP_POLY>, 32, 0);
    else if (tile == 8)
      e = backward ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_bwd_rows_persist<8, GP_EXP_POLY, false>, NB, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd_rows_persist<8, GP_EXP_POLY>, 32, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }
#define GP_OCC_F(T, C)                                                                                       \
  if (!backward && tile == T && chunk == C)                                                                  \
    e = row ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd_persist<T, C, GP_EXP_POLY_ROW>, \
                                                            (T / 8) * (T / 8) * 32, 0)                       \
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd_persist<T, C, GP_EXP_POLY>,     \
                                                            (T / 8) * (T / 8) * 32, 0);
#define GP_OCC_B(T, C)                                                                                       \
  if (backward && tile == T && chunk == C)                                                                   \
    e = row ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                 \
                  &n, k_raster_bwd_persist<T, C, GP_EXP_POLY_ROW, false>, (T / 8) * (T / 8) * 32, 0)        \
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                 \
                  &n, k_raster_bwd_persist<T, C, GP_EXP_POLY, false>, (T / 8) * (T / 8) * 32, 0);
  GP_OCC_F(16, 64) GP_OCC_F(16, 128) GP_OCC_F(16, 256) GP_OCC_F(8, 64) GP_OCC_F(8, 128) GP_OCC_F(8, 256)
  GP_OCC_B(16, 32) GP_OCC_B(16, 64) GP_OCC_B(16, 128) GP_OCC_B(8, 32) GP_OCC_B(8, 64) GP_OCC_B(8, 128)
#undef GP_OCC_F
#undef GP_OCC_B
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

GP_CHECK_READER(check_read_raster)

#ifdef GP_CHECK
__global__ void k_check_selftest(int i, int n) {
  if (threadIdx.x == 0) (void)GP_IN_RANGE(99, i, n);
}

void launch_check_selftest(cudaStream_t st) { k_check_selftest<<<1, 32, 0, st>>>(5, 4); }
#endif

}  // namespace gp
