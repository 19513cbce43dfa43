// raster_rows.cuh -- row-unit tile bodies of the default rasterisers (K-fwd and
// K-bwd with per-pixel exponentials, GP_EXP_POLY and GP_EXP_HW); included by
// raster.cu.
//
// One warp renders one (slice, tile).  The tile is cut into row segments of 8
// pixels: column band c (pixels 8c .. 8c + 7) of pixel row y, the tile's
// "buckets" b = c * TILE + y (32 of them for 16 x 16 tiles).  The warp takes
// the tile's binned Gaussians 32 at a time, one per lane.  A lane stages its
// Gaussian -- mu_2d and a~ of this slice (Eq. 9), the exponent's quadratic
// coefficients -- and, per column band, the exact range of pixel rows whose
// segment of pixel centres the culling ellipse d^T C d <= k^2 meets (the
// ellipse's height range over the band's strip).  Every (Gaussian, bucket) pair
// so found is a unit of 8 pixels, and only those are evaluated: a pixel row the
// ellipse misses costs nothing, unlike a whole 8 x 8 block or 8 x 4 half-block.
//
// The units of a round are listed in a fixed order -- bucket-major in the
// forward (the pixels they write), Gaussian-major in the backward (the
// Gaussian they differentiate) -- as the set bits of 32 words: word w lists,
// as a bit mask, the Gaussians of bucket w (forward) or the buckets of
// Gaussian w (backward).  Lane l takes the l-th contiguous run of R =
// ceil(N / 32) of the N units, so all lanes but the last few do the same
// number.  Consecutive units of a run mostly share their word: a lane
// accumulates in registers and writes out when the word changes ("a piece").
// A piece that neither starts nor ends a run belongs to the lane alone and is
// written directly; the first and last pieces of a run may continue in the
// neighbouring lanes' runs, so they are kept in per-lane slots and, after the
// round, the owner of each word sums its pieces in lane order.  Every sum has
// a fixed order, so results are bitwise reproducible, and there is no block
// barrier at all.
//
// Along a unit's row the exponent is A + B q + C q^2 in the offset q = p - 3.5
// of pixel p from the band's centre column.  The pixels are taken in mirrored
// couples (q, -q), which share A + C q^2, two pixels per packed fp32x2
// instruction.
#pragma once

namespace gp {

constexpr int kRowGauss = 32;  // Gaussians per staging round: one per lane

// One staged Gaussian of the row-unit bodies.
struct RowGauss {
  float mx, my;      // mu_2d of this slice, tile-relative
  float c0, c1, c2;  // exponent (log2 units): c0 dx^2 + c1 dx dy + c2 dy^2 = -log2(e)/2 d^T C d
  float at;          // a~ = A opacity_r (Eq. 9), or alpha opacity on a voxelizer plane
  float C00, C01, C11, d, w;  // the backward's fold: conic, delta, opacity_r
  unsigned mask;     // buckets (bit c * TILE + y) whose segment the culling ellipse meets
};

// Stages Gaussian g for slice position zsv of the tile at (x0, y0); nrows /
// nbands: the tile's rows and column bands inside the image.  On a voxelizer
// plane the culling ellipse is the plane's section of the 3D one, d^T C d <=
// k2 - delta^2 / Sigma_zz (its extents scaled to match).
template <int EXPM, int TILE>
__device__ __forceinline__ RowGauss stage_rows(const SliceRec* __restrict__ rec, uint32_t g, float zsv, float x0,
                                               float y0, float k2, bool vox, int nrows, int nbands) {
  const float4* rp = reinterpret_cast<const float4*>(rec + g);
  const float4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2), r3 = __ldg(rp + 3);
  RowGauss o;
  o.d = r0.z - zsv;
  o.w = exp2_sel<EXPM>(fmaxf(-0.5f * kLog2e * o.d * o.d * r0.w, kExpFloor));
  o.mx = (r0.x - x0) - r1.x * o.d;
  o.my = (r0.y - y0) - r1.y * o.d;
  o.C00 = r2.x;
  o.C01 = r2.y;
  o.C11 = r2.z;
  o.c0 = -0.5f * kLog2e * o.C00;
  o.c1 = -kLog2e * o.C01;
  o.c2 = -0.5f * kLog2e * o.C11;
  o.at = r1.z * o.w;
  o.mask = row_unit_mask<TILE>(r0, r2, r3, o.d, o.mx, o.my, k2, vox, nrows, nbands);
  return o;
}

// Transposes the 32 x 32 bit matrix whose row l is lane l's word: afterwards
// lane b holds bit j = bit b of lane j's word.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
  const unsigned m[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int s = 16 >> k;
    const unsigned y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~m[k]) | ((y & ~m[k]) >> s)) : ((x & m[k]) | ((y & m[k]) << s));
  }
  return x;
}

// Position of the k-th (from 0) set bit of x; x has more than k set bits.
__device__ __forceinline__ int select_bit(unsigned x, int k) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const int c = __popc(x & ((1u << s) - 1u));
    if (c <= k) {
      k -= c;
      x >>= s;
      pos += s;
    }
  }
  return pos;
}

// Shared state of one round's unit list: the 32 words, their exclusive prefix
// counts of set bits (pre[32] = N) and the per-lane first / last pieces.
template <int NV>
struct RunSmem {
  unsigned words[32];
  int pre[33];
  int nxt[32];  // the next word with a set bit after word w (32 if none)
  float4 head[32][NV];
  float4 tail[32][NV];
};

// Stores lane `lane`'s word with the prefix counts and next-nonempty-word
// links of all 32 (the caller syncs the warp before reading them).
template <int NV>
__device__ __forceinline__ void run_publish(RunSmem<NV>& rs, unsigned word, int lane) {
  const int c = __popc(word);
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int sh = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += sh;
  }
  const unsigned busy = __ballot_sync(0xffffffffu, word != 0u);
  const unsigned later = lane == 31 ? 0u : busy & (0xfffffffeu << lane);
  rs.words[lane] = word;
  rs.pre[lane] = incl - c;
  rs.nxt[lane] = later ? __ffs(later) - 1 : 32;
  if (lane == 31) rs.pre[32] = incl;
}

// Lane `lane`'s run of the round: its first unit's word and the remaining set
// bits of that word from that unit on; R units per run, N in all.
struct RunStart {
  int i0, n;      // first unit index, number of units of this lane
  int w;          // word of the first unit
  unsigned rem;   // set bits of word w from the first unit on
};

template <int NV>
__device__ __forceinline__ RunStart run_start(const RunSmem<NV>& rs, int R, int lane) {
  RunStart r;
  const int N = rs.pre[32];
  r.i0 = lane * R;
  r.n = max(0, min(N - r.i0, R));
  r.w = 0;
  r.rem = 0u;
  if (r.n > 0) {
    // the largest w with pre[w] <= i0 (its word holds unit i0)
    int w = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
      if (w + s < 32 && rs.pre[w + s] <= r.i0) w += s;
    r.w = w;
    const unsigned x = rs.words[w];
    const int p = select_bit(x, r.i0 - rs.pre[w]);
    r.rem = x & ~((1u << p) - 1u);
  }
  return r;
}

// Where the pieces of word w lie: pieces in lanes [llo, lhi]; own = true when
// its only piece sits inside one run without starting or ending it (then the
// lane has written it itself).  For each lane l of the range, the piece is the
// lane's last (tail slot) when the word's units reach the run's end, else its
// first (head slot).
struct WordPieces {
  int llo, lhi;
  bool any, own;
};

template <int NV>
__device__ __forceinline__ WordPieces word_pieces(const RunSmem<NV>& rs, int R, int w) {
  WordPieces p;
  const int e0 = rs.pre[w], e1 = rs.pre[w + 1], N = rs.pre[32];
  p.any = e1 > e0;
  p.llo = p.any ? e0 / R : 0;
  p.lhi = p.any ? (e1 - 1) / R : -1;
  p.own = p.any && p.llo == p.lhi && e0 > p.llo * R && e1 < min(N, (p.llo + 1) * R);
  return p;
}

template <int NV>
__device__ __forceinline__ bool piece_is_tail(const RunSmem<NV>& rs, int R, int w, int l) {
  return rs.pre[w + 1] >= min(rs.pre[32], (l + 1) * R);
}

// ------------------------------------------------------------- forward

template <int TILE>
struct RowFwdSmem {
  float4 g0[kRowGauss];  // (mx, my, c0, c1)
  float2 g1[kRowGauss];  // (c2, a~)
  alignas(16) float img[TILE * TILE / 8][8];  // per bucket: its 8 pixels, summed over the rounds so far
  RunSmem<2> rs;
};

// Forward of one (slice s, tile t) of item a: every pixel of the tile is written.
template <int TILE, int EXPM>
__device__ __forceinline__ void fwd_tile_rows(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                              const uint32_t* __restrict__ vals,
                                              const uint32_t* __restrict__ emit_gid,
                                              const uint2* __restrict__ ranges, RowFwdSmem<TILE>& sm) {
  constexpr int NB = TILE * TILE / 8;  // buckets
  const int T = a.TX * a.TY;
  if (!GP_IN_RANGE(6, local_key, T * a.S)) return;
  const int lane = threadIdx.x & 31;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const int nrows = min(TILE, a.H - ty * TILE), nbands = min(TILE / 8, (a.W - tx * TILE + 7) >> 3);
  const float zsv = a.zorig[s];
  for (int b = lane; b < NB; b += 32) {
    reinterpret_cast<float4*>(sm.img[b])[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(sm.img[b])[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (uint32_t base = rg.x; base < rg.y; base += kRowGauss) {
    const int cnt = (int)min((uint32_t)kRowGauss, rg.y - base);
    // stage one Gaussian per lane
    unsigned mask = 0u;
    if (lane < cnt) {
      const uint32_t v = vals[base + lane];
      const uint32_t g = emit_gid ? emit_gid[v] : v;  // sorted values: emission indices, or Gaussian ids
      if (GP_IN_RANGE(5, (int64_t)g - a.gbase, a.n)) {
        const RowGauss q = stage_rows<EXPM, TILE>(rec, g, zsv, x0, y0, a.k2, a.vox != 0, nrows, nbands);
        sm.g0[lane] = make_float4(q.mx, q.my, q.c0, q.c1);
        sm.g1[lane] = make_float2(q.c2, q.at);
        mask = q.mask;
      }
    }
    // bucket-major unit list: word b = the Gaussians that meet bucket b
    run_publish(sm.rs, warp_transpose32(mask, lane), lane);
    __syncwarp();
    const int N = sm.rs.pre[32];
    if (N > 0) {
      const int R = (N + 31) >> 5;
      RunStart st = run_start(sm.rs, R, lane);
      int w = st.w;
      unsigned rem = st.rem;
      bool first = true;
      float2 a01 = make_float2(0.f, 0.f), a23 = a01, a54 = a01, a76 = a01;
      for (int k = 0; k < R; ++k) {
        const bool act = k < st.n;
        if (act && rem == 0u) {
          // the run moves on to the next bucket: the piece of bucket w ends here
          if (first) {
            sm.rs.head[lane][0] = make_float4(a01.x, a01.y, a23.x, a23.y);
            sm.rs.head[lane][1] = make_float4(a54.y, a54.x, a76.y, a76.x);
          } else if (GP_IN_RANGE(9, w, NB)) {
            float4* o = reinterpret_cast<float4*>(sm.img[w]);
            const float4 p0 = o[0], p1 = o[1];
            o[0] = make_float4(p0.x + a01.x, p0.y + a01.y, p0.z + a23.x, p0.w + a23.y);
            o[1] = make_float4(p1.x + a54.y, p1.y + a54.x, p1.z + a76.y, p1.w + a76.x);
          }
          first = false;
          a01 = a23 = a54 = a76 = make_float2(0.f, 0.f);
          w = sm.rs.nxt[w];
          rem = GP_IN_RANGE(10, w, 32) ? sm.rs.words[w] : 0xffffffffu;
        }
        if (act) {
          const int j = __ffs(rem) - 1;
          rem &= rem - 1u;
          const float4 g0 = sm.g0[j];
          const float2 g1 = sm.g1[j];
          const int cb = w / TILE, y = w - cb * TILE;
          const float dxc = (float)(8 * cb) + 4.0f - g0.x;
          const float dy = (float)y + 0.5f - g0.y;
          const float u = g0.w * dy;
          const float A = fmaf(dxc, fmaf(g0.z, dxc, u), g1.x * dy * dy);
          const float B = fmaf(2.0f * g0.z, dxc, u);
          const float2 A2 = make_float2(A, A), C2 = make_float2(g0.z, g0.z);
          const float2 B2 = make_float2(B, B), at2 = make_float2(g1.y, g1.y);
          // couples (q, -q): pixels (0, 1) with (7, 6), q = (-3.5, -2.5); (2, 3) with (5, 4), q = (-1.5, -0.5)
          const float2 bA = __ffma2_rn(C2, make_float2(12.25f, 6.25f), A2);
          const float2 bB = __ffma2_rn(C2, make_float2(2.25f, 0.25f), A2);
          a01 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(-3.5f, -2.5f), bA), a01);
          a76 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(3.5f, 2.5f), bA), a76);
          a23 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(-1.5f, -0.5f), bB), a23);
          a54 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(1.5f, 0.5f), bB), a54);
        }
      }
      if (st.n > 0) {
        sm.rs.tail[lane][0] = make_float4(a01.x, a01.y, a23.x, a23.y);
        sm.rs.tail[lane][1] = make_float4(a54.y, a54.x, a76.y, a76.x);
      }
      __syncwarp();
      // the owner of each bucket adds its shared pieces in lane order
      for (int b = lane; b < NB; b += 32) {
        const WordPieces p = word_pieces(sm.rs, R, b);
        if (p.any && !p.own) {
          float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
          for (int l = p.llo; l <= p.lhi; ++l) {
            if (!GP_IN_RANGE(11, l, 32)) break;
            const bool tl = piece_is_tail(sm.rs, R, b, l);
            const float4 q0 = tl ? sm.rs.tail[l][0] : sm.rs.head[l][0];
            const float4 q1 = tl ? sm.rs.tail[l][1] : sm.rs.head[l][1];
            s0 = make_float4(s0.x + q0.x, s0.y + q0.y, s0.z + q0.z, s0.w + q0.w);
            s1 = make_float4(s1.x + q1.x, s1.y + q1.y, s1.z + q1.z, s1.w + q1.w);
          }
          float4* o = reinterpret_cast<float4*>(sm.img[b]);
          const float4 p0 = o[0], p1 = o[1];
          o[0] = make_float4(p0.x + s0.x, p0.y + s0.y, p0.z + s0.z, p0.w + s0.w);
          o[1] = make_float4(p1.x + s1.x, p1.y + s1.y, p1.z + s1.z, p1.w + s1.w);
        }
      }
    }
    __syncwarp();
  }
  // write the tile: lane b writes bucket b's 8 pixels
  for (int b = lane; b < NB; b += 32) {
    const int cb = b / TILE, y = b - cb * TILE;
    const int py = ty * TILE + y, px0 = tx * TILE + 8 * cb;
    if (py >= a.H || px0 >= a.W) continue;
    const float4 p0 = reinterpret_cast<const float4*>(sm.img[b])[0];
    const float4 p1 = reinterpret_cast<const float4*>(sm.img[b])[1];
    float* o = a.out + ((int64_t)s * a.H + py) * a.W + px0;
    if (px0 + 8 <= a.W && ((((uintptr_t)o) & 15u) == 0)) {
      reinterpret_cast<float4*>(o)[0] = p0;
      reinterpret_cast<float4*>(o)[1] = p1;
    } else {
      const float v[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (px0 + p < a.W) o[p] = v[p];
    }
  }
}

// ------------------------------------------------------ forward, 16 x 16

// For 16 x 16 tiles the warp's 32 lanes match the tile's 32 row segments, so
// the forward lets each lane own one: lane b keeps its 8 pixels in registers
// for the whole tile and walks, in ascending list order, the Gaussians whose
// culling ellipse meets its segment.  Nothing is handed between lanes, every
// pixel is summed over its Gaussians in list order (ascending Gaussian id),
// and a lane's work is its own segment's list: rounds of kOwnGauss Gaussians
// (eight groups of 32) keep the lanes' list lengths close (about 0.9 of the
// longest on the fit step's tiles).
constexpr int kOwnGauss = 256;

struct OwnFwdSmem {
  float4 g0[kOwnGauss];  // (mx, my, c0, c1)
  float2 g1[kOwnGauss];  // (c2, a~)
  unsigned words[kOwnGauss / 32][32];  // [group][segment]: the group's Gaussians that meet the segment
};

template <int EXPM>
__device__ __forceinline__ void fwd_tile_owner(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                               const uint32_t* __restrict__ vals,
                                               const uint32_t* __restrict__ emit_gid,
                                               const uint2* __restrict__ ranges, OwnFwdSmem& sm) {
  constexpr int TILE = 16;
  const int T = a.TX * a.TY;
  if (!GP_IN_RANGE(6, local_key, T * a.S)) return;
  const int lane = threadIdx.x & 31;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const int nrows = min(TILE, a.H - ty * TILE), nbands = min(TILE / 8, (a.W - tx * TILE + 7) >> 3);
  const float zsv = a.zorig[s];
  // this lane's segment: column band cb, pixel row y
  const int cb = lane >> 4, y = lane & 15;
  const float fx = (float)(8 * cb) + 4.0f, fy = (float)y + 0.5f;
  float2 a01 = make_float2(0.f, 0.f), a23 = a01, a54 = a01, a76 = a01;
  for (uint32_t base = rg.x; base < rg.y; base += kOwnGauss) {
    const int cnt = (int)min((uint32_t)kOwnGauss, rg.y - base);
    const int ngroups = (cnt + 31) >> 5;
    for (int gi = 0; gi < ngroups; ++gi) {
      const int j = gi * 32 + lane;
      unsigned mask = 0u;
      if (j < cnt) {
        const uint32_t v = vals[base + j];
        const uint32_t g = emit_gid ? emit_gid[v] : v;  // sorted values: emission indices, or Gaussian ids
        if (GP_IN_RANGE(5, (int64_t)g - a.gbase, a.n)) {
          const RowGauss q = stage_rows<EXPM, TILE>(rec, g, zsv, x0, y0, a.k2, a.vox != 0, nrows, nbands);
          sm.g0[j] = make_float4(q.mx, q.my, q.c0, q.c1);
          sm.g1[j] = make_float2(q.c2, q.at);
          mask = q.mask;
        }
      }
      sm.words[gi][lane] = warp_transpose32(mask, lane);
    }
    __syncwarp();
    int gi = 0;
    unsigned rem = sm.words[0][lane];
    for (;;) {
      while (rem == 0u && gi + 1 < ngroups) {
        ++gi;
        rem = sm.words[gi][lane];
      }
      if (rem == 0u) break;
      const int j = gi * 32 + __ffs(rem) - 1;
      rem &= rem - 1u;
      const float4 g0 = sm.g0[j];
      const float2 g1 = sm.g1[j];
      const float dxc = fx - g0.x, dy = fy - g0.y;
      const float u = g0.w * dy;
      const float A = fmaf(dxc, fmaf(g0.z, dxc, u), g1.x * dy * dy);
      const float B = fmaf(2.0f * g0.z, dxc, u);
      const float2 A2 = make_float2(A, A), C2 = make_float2(g0.z, g0.z);
      const float2 B2 = make_float2(B, B), at2 = make_float2(g1.y, g1.y);
      // couples (q, -q): pixels (0, 1) with (7, 6), q = (-3.5, -2.5); (2, 3) with (5, 4), q = (-1.5, -0.5)
      const float2 bA = __ffma2_rn(C2, make_float2(12.25f, 6.25f), A2);
      const float2 bB = __ffma2_rn(C2, make_float2(2.25f, 0.25f), A2);
      a01 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(-3.5f, -2.5f), bA), a01);
      a76 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(3.5f, 2.5f), bA), a76);
      a23 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(-1.5f, -0.5f), bB), a23);
      a54 = __ffma2_rn(at2, couple_exp2<EXPM>(B2, make_float2(1.5f, 0.5f), bB), a54);
    }
    __syncwarp();
  }
  const int py = ty * TILE + y, px0 = tx * TILE + 8 * cb;
  if (py >= a.H || px0 >= a.W) return;
  float* o = a.out + ((int64_t)s * a.H + py) * a.W + px0;
  if (px0 + 8 <= a.W && ((((uintptr_t)o) & 15u) == 0)) {
    reinterpret_cast<float4*>(o)[0] = make_float4(a01.x, a01.y, a23.x, a23.y);
    reinterpret_cast<float4*>(o)[1] = make_float4(a54.y, a54.x, a76.y, a76.x);
  } else {
    const float v[8] = {a01.x, a01.y, a23.x, a23.y, a54.y, a54.x, a76.y, a76.x};
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (px0 + p < a.W) o[p] = v[p];
  }
}

// ------------------------------------------------------------- backward

template <int TILE>
struct RowBwdSmem {
  static constexpr int GS = 12;  // floats per bucket row of dL/dI (8 + 4 of padding: rows fall in different banks)
  alignas(16) float G[TILE * TILE / 8 * GS];  // per bucket: pixels 0, 1, 2, 3, 7, 6, 5, 4 of its segment
  float4 g0[kRowGauss];  // (mx, my, c0, c1)
  float4 g1[kRowGauss];  // (c2, a~, C00, C01)
  float4 g2[kRowGauss];  // (C11, delta, opacity_r, Gaussian id as bits)
  float4 acc[kRowGauss][2];  // per Gaussian: its six moments (and two unused)
  RunSmem<2> rs;
};

// Backward of one (slice s, tile t) of item a.  Per Gaussian the units sum the
// six moments sum G E {1, dx, dy, dx^2, dx dy, dy^2} (E the Gaussian's
// exponential, G = dL/dI, d = pixel - mu_2d), which are folded into its 10
// accumulators (atomics) or written as a per-pair partial (deterministic mode).
template <int TILE, int EXPM, bool DET>
__device__ __forceinline__ void bwd_tile_rows(const SliceArgs& a, int local_key, const SliceRec* __restrict__ rec,
                                              const uint32_t* __restrict__ vals,
                                              const uint32_t* __restrict__ emit_gid,
                                              const uint2* __restrict__ ranges, float* __restrict__ accum,
                                              float4* __restrict__ partial, RowBwdSmem<TILE>& sm) {
  constexpr int GS = RowBwdSmem<TILE>::GS;
  const int T = a.TX * a.TY;
  if (!GP_IN_RANGE(6, local_key, T * a.S)) return;
  const uint2 rg = ranges[a.key_base + (uint32_t)local_key];
  if (rg.y <= rg.x) return;  // uniform over the warp
  const int lane = threadIdx.x & 31;
  const int s = local_key / T, t = local_key - s * T;
  const int ty = t / a.TX, tx = t - ty * a.TX;
  const float x0 = (float)(tx * TILE), y0 = (float)(ty * TILE);
  const int nrows = min(TILE, a.H - ty * TILE), nbands = min(TILE / 8, (a.W - tx * TILE + 7) >> 3);
  const float zsv = a.zorig[s];
  // the tile's dL/dI (zero outside the image), bucket by bucket, each row's
  // second half mirrored so that both halves of a couple are 16-byte loads
  for (int i = lane; i < TILE * TILE; i += 32) {
    const int yy = i / TILE, xx = i - yy * TILE;
    const int py = ty * TILE + yy, px = tx * TILE + xx;
    const int cx = xx & 7;
    const float gv = (py < a.H && px < a.W) ? a.dL_dI[((int64_t)s * a.H + py) * a.W + px] : 0.0f;
    sm.G[((xx >> 3) * TILE + yy) * GS + (cx < 4 ? cx : 11 - cx)] = gv;
  }
  __syncwarp();
  for (uint32_t base = rg.x; base < rg.y; base += kRowGauss) {
    const int cnt = (int)min((uint32_t)kRowGauss, rg.y - base);
    unsigned mask = 0u;
    if (lane < cnt) {
      const uint32_t v = vals[base + lane];
      const uint32_t g = emit_gid ? emit_gid[v] : v;  // sorted values: emission indices, or Gaussian ids
      if (GP_IN_RANGE(5, (int64_t)g - a.gbase, a.n)) {
        const RowGauss q = stage_rows<EXPM, TILE>(rec, g, zsv, x0, y0, a.k2, a.vox != 0, nrows, nbands);
        sm.g0[lane] = make_float4(q.mx, q.my, q.c0, q.c1);
        sm.g1[lane] = make_float4(q.c2, q.at, q.C00, q.C01);
        sm.g2[lane] = make_float4(q.C11, q.d, q.w, __uint_as_float(g));
        mask = q.mask;
      }
      sm.acc[lane][0] = make_float4(0.f, 0.f, 0.f, 0.f);
      sm.acc[lane][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // Gaussian-major unit list: word j = the buckets Gaussian j meets
    run_publish(sm.rs, mask, lane);
    __syncwarp();
    const int N = sm.rs.pre[32];
    const int R = (N + 31) >> 5;
    if (N > 0) {
      RunStart st = run_start(sm.rs, R, lane);
      int w = st.w;
      unsigned rem = st.rem;
      bool first = true;
      float M0 = 0.f, M1 = 0.f, M2 = 0.f, M3 = 0.f, M4 = 0.f, M5 = 0.f;
      float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f);
      float c2 = 0.f;
      if (st.n > 0) {
        g0 = sm.g0[w];
        c2 = sm.g1[w].x;
      }
      for (int k = 0; k < R; ++k) {
        const bool act = k < st.n;
        if (act && rem == 0u) {
          // the run moves on to the next Gaussian: the piece of Gaussian w ends here, into the
          // lane's head slot (its first piece) or the Gaussian's own accumulators
          float4* dst = first ? sm.rs.head[lane] : sm.acc[GP_IN_RANGE(12, w, kRowGauss) ? w : 0];
          dst[0] = make_float4(M0, M1, M2, M3);
          dst[1] = make_float4(M4, M5, 0.f, 0.f);
          first = false;
          M0 = M1 = M2 = M3 = M4 = M5 = 0.f;
          w = sm.rs.nxt[w];
          if (!GP_IN_RANGE(10, w, 32)) w = 31;
          rem = sm.rs.words[w];
          g0 = sm.g0[w];
          c2 = sm.g1[w].x;
        }
        if (act) {
          const int b = __ffs(rem) - 1;
          rem &= rem - 1u;
          const int cb = b / TILE, y = b - cb * TILE;
          const float dxc = (float)(8 * cb) + 4.0f - g0.x;
          const float dy = (float)y + 0.5f - g0.y;
          const float u = g0.w * dy;
          const float A = fmaf(dxc, fmaf(g0.z, dxc, u), c2 * dy * dy);
          const float B = fmaf(2.0f * g0.z, dxc, u);
          const float2 A2 = make_float2(A, A), C2 = make_float2(g0.z, g0.z), B2 = make_float2(B, B);
          const float* Gr = sm.G + b * GS;
          const float4 gx = *reinterpret_cast<const float4*>(Gr);      // pixels 0, 1, 2, 3 (q < 0)
          const float4 gy = *reinterpret_cast<const float4*>(Gr + 4);  // pixels 7, 6, 5, 4 (their mirrors)
          // with X = G E at the q < 0 pixels and Y at their mirrors:
          //   sum G E = X + Y,  sum q G E = q (X + Y) - 2 q Y,  sum q^2 G E = q^2 (X + Y)
          const float2 bA = __ffma2_rn(C2, make_float2(12.25f, 6.25f), A2);
          const float2 bB = __ffma2_rn(C2, make_float2(2.25f, 0.25f), A2);
          const float2 qA = make_float2(-3.5f, -2.5f), qB = make_float2(-1.5f, -0.5f);
          const float2 YA = __fmul2_rn(make_float2(gy.x, gy.y), couple_exp2<EXPM, true, true>(B2, make_float2(3.5f, 2.5f), bA));
          const float2 XA = __ffma2_rn(make_float2(gx.x, gx.y), couple_exp2<EXPM, true, true>(B2, qA, bA), YA);
          const float2 YB = __fmul2_rn(make_float2(gy.z, gy.w), couple_exp2<EXPM, true, true>(B2, make_float2(1.5f, 0.5f), bB));
          const float2 XB = __ffma2_rn(make_float2(gx.z, gx.w), couple_exp2<EXPM, true, true>(B2, qB, bB), YB);
          const float2 P0 = __fadd2_rn(XA, XB);
          float2 P1 = __ffma2_rn(qB, XB, __fmul2_rn(qA, XA));
          P1 = __ffma2_rn(make_float2(7.0f, 5.0f), YA, P1);
          P1 = __ffma2_rn(make_float2(3.0f, 1.0f), YB, P1);
          const float2 P2 = __ffma2_rn(make_float2(2.25f, 0.25f), XB, __fmul2_rn(make_float2(12.25f, 6.25f), XA));
          const float S0 = P0.x + P0.y, S1 = P1.x + P1.y, S2 = P2.x + P2.y;
          // moments in d = (dxc + q, dy)
          const float t1 = fmaf(dxc, S0, S1);  // sum dx G E
          const float t3 = dy * S0;            // sum dy G E
          M0 += S0;
          M1 += t1;
          M2 += t3;
          M3 += fmaf(dxc, t1, fmaf(dxc, S1, S2));
          M4 = fmaf(dy, t1, M4);
          M5 = fmaf(dy, t3, M5);
        }
      }
      if (st.n > 0) {
        sm.rs.tail[lane][0] = make_float4(M0, M1, M2, M3);
        sm.rs.tail[lane][1] = make_float4(M4, M5, 0.f, 0.f);
      }
    }
    __syncwarp();
    // the owner of each Gaussian sums its shared pieces in lane order, then folds
    if (lane < cnt) {
      float4 m0 = sm.acc[lane][0], m1 = sm.acc[lane][1];
      if (N > 0) {
        const WordPieces p = word_pieces(sm.rs, R, lane);
        if (p.any && !p.own) {
          m0 = make_float4(0.f, 0.f, 0.f, 0.f);
          m1 = m0;
          for (int l = p.llo; l <= p.lhi; ++l) {
            if (!GP_IN_RANGE(11, l, 32)) break;
            const bool tl = piece_is_tail(sm.rs, R, lane, l);
            const float4 q0 = tl ? sm.rs.tail[l][0] : sm.rs.head[l][0];
            const float4 q1 = tl ? sm.rs.tail[l][1] : sm.rs.head[l][1];
            m0 = make_float4(m0.x + q0.x, m0.y + q0.y, m0.z + q0.z, m0.w + q0.w);
            m1 = make_float4(m1.x + q1.x, m1.y + q1.y, 0.f, 0.f);
          }
        }
      }
      const float4 g1 = sm.g1[lane], g2 = sm.g2[lane];
      const float at = g1.y, C00 = g1.z, C01 = g1.w, C11 = g2.x;
      // dE/dmu_2d = E C d; dE/dC00 = -E dx^2/2, dE/dC01 = -E dx dy, dE/dC11 = -E dy^2/2
      const float g_at = m0.x;
      const float gmx = at * (C00 * m0.y + C01 * m0.z);
      const float gmy = at * (C01 * m0.y + C11 * m0.z);
      const float gc00 = -0.5f * at * m0.w;
      const float gc01 = -at * m1.x;
      const float gc11 = -0.5f * at * m1.y;
      const float d = g2.y, w = g2.z;
      if constexpr (DET) {
        const uint32_t e = vals[base + lane];
        partial[2 * (size_t)e] = make_float4(g_at, gmx, gmy, gc00);
        partial[2 * (size_t)e + 1] = make_float4(gc01, gc11, d, w);
      } else if (N > 0 && sm.rs.pre[lane + 1] > sm.rs.pre[lane]) {
        // a Gaussian with no unit on this tile adds nothing
        float* A = accum + (size_t)__float_as_uint(g2.w) * ACC10;
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
