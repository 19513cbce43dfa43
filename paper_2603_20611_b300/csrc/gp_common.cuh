// gp_common.cuh -- shared device helpers of the sm_103a slice projection library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gp.h"

namespace gp {

// log2(e) as an fp32 literal of the mathematical constant.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kExpFloor = -125.0f;  // 2^-125 ~ 2.4e-38: below fp32 resolution of any sum

// ---------------------------------------------------------------- exp2
// 2^x = 2^n 2^f, n = round(x), f = x - n in [-1/2, 1/2]; 2^f by a degree-6
// polynomial with p(0) = 1 fitted for minimal relative error on [-1/2, 1/2]
// (Remez exchange; coefficients derived by csrc/exp2_poly.py, max relative
// error 1.9 ulp of 2^-24 with plain fp32 Horner).  n is recovered with the
// round-to-nearest trick (x + 1.5*2^23 leaves n in the low mantissa bits) and
// inserted into the exponent with an integer shift-add.  Valid for
// x in [-125, 0.5]; callers clamp below.
#define GP_EXP2_C1 0.6931472420692444f
#define GP_EXP2_C2 0.24022652208805084f
#define GP_EXP2_C3 0.055503103882074356f
#define GP_EXP2_C4 0.009617692790925503f
#define GP_EXP2_C5 0.0013406643411144614f
#define GP_EXP2_C6 0.00015594677824992687f

__device__ __forceinline__ float exp2_poly(float x) {
  const float kShift = 12582912.0f;  // 1.5 * 2^23
  float t = __fadd_rn(x, kShift);
  float n = __fsub_rn(t, kShift);
  float f = __fsub_rn(x, n);
  float p = GP_EXP2_C6;
  p = fmaf(p, f, GP_EXP2_C5);
  p = fmaf(p, f, GP_EXP2_C4);
  p = fmaf(p, f, GP_EXP2_C3);
  p = fmaf(p, f, GP_EXP2_C2);
  p = fmaf(p, f, GP_EXP2_C1);
  p = fmaf(p, f, 1.0f);
  return __int_as_float(__float_as_int(p) + (__float_as_int(t) << 23));
}

// exp2_poly on two values at once with the packed fp32x2 instructions of
// sm_100-class SMs (one instruction issues both lanes' add / fma): the same
// operations, each rounded exactly as in exp2_poly, so the results are
// bitwise those of two exp2_poly calls.
__device__ __forceinline__ float2 exp2_poly2(float2 x) {
  const float kShift = 12582912.0f;  // 1.5 * 2^23
  const float2 t = __fadd2_rn(x, make_float2(kShift, kShift));
  const float2 n = __fadd2_rn(t, make_float2(-kShift, -kShift));
  const float2 f = __ffma2_rn(n, make_float2(-1.0f, -1.0f), x);  // x - n, rounded once
  float2 p = make_float2(GP_EXP2_C6, GP_EXP2_C6);
  p = __ffma2_rn(p, f, make_float2(GP_EXP2_C5, GP_EXP2_C5));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2_C4, GP_EXP2_C4));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2_C3, GP_EXP2_C3));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2_C2, GP_EXP2_C2));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2_C1, GP_EXP2_C1));
  p = __ffma2_rn(p, f, make_float2(1.0f, 1.0f));
  return make_float2(__int_as_float(__float_as_int(p.x) + (__float_as_int(t.x) << 23)),
                     __int_as_float(__float_as_int(p.y) + (__float_as_int(t.y) << 23)));
}

// The backward's exponential: the same range reduction and exponent insert
// with a degree-4 polynomial (Remez, p(0) = 1, csrc/exp2_poly.py; max
// relative error 3.6e-6 on the reduced range with fp32 Horner).  The backward
// recomputes every pixel's exponential only to weight dL/dI in the gradient
// sums, which are held to 1e-3 relative; the images keep the degree-6 form.
#define GP_EXP2G_C1 0.6931136250495911f
#define GP_EXP2G_C2 0.24020710587501526f
#define GP_EXP2G_C3 0.055976882576942444f
#define GP_EXP2G_C4 0.009782912209630013f

__device__ __forceinline__ float exp2_grad(float x) {
  const float kShift = 12582912.0f;  // 1.5 * 2^23
  float t = __fadd_rn(x, kShift);
  float n = __fsub_rn(t, kShift);
  float f = __fsub_rn(x, n);
  float p = GP_EXP2G_C4;
  p = fmaf(p, f, GP_EXP2G_C3);
  p = fmaf(p, f, GP_EXP2G_C2);
  p = fmaf(p, f, GP_EXP2G_C1);
  p = fmaf(p, f, 1.0f);
  return __int_as_float(__float_as_int(p) + (__float_as_int(t) << 23));
}

// exp2_grad on two values per packed instruction, bitwise the scalar form.
__device__ __forceinline__ float2 exp2_grad2(float2 x) {
  const float kShift = 12582912.0f;  // 1.5 * 2^23
  const float2 t = __fadd2_rn(x, make_float2(kShift, kShift));
  const float2 n = __fadd2_rn(t, make_float2(-kShift, -kShift));
  const float2 f = __ffma2_rn(n, make_float2(-1.0f, -1.0f), x);  // x - n, rounded once
  float2 p = make_float2(GP_EXP2G_C4, GP_EXP2G_C4);
  p = __ffma2_rn(p, f, make_float2(GP_EXP2G_C3, GP_EXP2G_C3));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2G_C2, GP_EXP2G_C2));
  p = __ffma2_rn(p, f, make_float2(GP_EXP2G_C1, GP_EXP2G_C1));
  p = __ffma2_rn(p, f, make_float2(1.0f, 1.0f));
  return make_float2(__int_as_float(__float_as_int(p.x) + (__float_as_int(t.x) << 23)),
                     __int_as_float(__float_as_int(p.y) + (__float_as_int(t.y) << 23)));
}

// The SFU instruction, as a benchmarked alternative (GP_EXP_HW).
__device__ __forceinline__ float exp2_hw(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int MODE>
__device__ __forceinline__ float exp2_sel(float x) {
  if constexpr (MODE == GP_EXP_HW) return exp2_hw(x);
  else return exp2_poly(x);
}

template <int MODE>
__device__ __forceinline__ float2 exp2_sel2(float2 x) {
  if constexpr (MODE == GP_EXP_HW) return make_float2(exp2_hw(x.x), exp2_hw(x.y));
  else return exp2_poly2(x);
}

// The backward's per-pixel exponentials: exp2_grad for the polynomial modes.
template <int MODE>
__device__ __forceinline__ float exp2_sel_grad(float x) {
  if constexpr (MODE == GP_EXP_HW) return exp2_hw(x);
  else return exp2_grad(x);
}

template <int MODE>
__device__ __forceinline__ float2 exp2_sel2_grad(float2 x) {
  if constexpr (MODE == GP_EXP_HW) return make_float2(exp2_hw(x.x), exp2_hw(x.y));
  else return exp2_grad2(x);
}

// Exponentials of two consecutive samples (2p, 2p + 1) of a row: e = A + B q +
// C q^2 floored at kExpFloor, two samples per packed fp32x2 instruction (each
// rounded as the scalar form rounds it).
template <int EXPM>
__device__ __forceinline__ float2 pair_exp2(float2 C2, float2 B2, float2 A2, float2 q) {
  float2 e = __ffma2_rn(__ffma2_rn(C2, q, B2), q, A2);
  e.x = fmaxf(e.x, kExpFloor);
  e.y = fmaxf(e.y, kExpFloor);
  return exp2_sel2<EXPM>(e);
}



// ------------------------------------------------------------ row units
// Culling cells are widened by this many pixels so that rounding only ever
// adds cells (an extra cell adds pixels where every term is below eps).
constexpr float kCellTol = 1e-3f;

// Rows [lo, hi] (tile-relative, lo > hi when none) whose pixel-centre segment
// x in [xa, xb] (tile-relative) the ellipse d^T C d <= k2 meets; (mx, my) the
// tile-relative centre, rx / ry its half-extents, inv00 = 1 / C00, inv11 =
// 1 / C11.  At dx from the centre the ellipse's vertical chord is centred on
// -(C01 / C11) dx with half-height h(dx) = sqrt((k2 / C11)(1 - dx^2 / rx^2)).
// The upper edge -(C01/C11) dx + h(dx) is concave, so over the strip it is
// highest at the strip point nearest the ellipse's topmost point, dx_t =
// -(C01 / C00) ry; the lower edge, convex, is lowest nearest -dx_t.  The range
// is widened by kCellTol so that rounding only ever adds rows; that widening
// also covers the approximate reciprocal and square roots (a few ulp).
__device__ __forceinline__ void band_rows(float C01, float inv00, float inv11, float rx, float ry, float k2,
                                          float mx, float my, float xa, float xb, int nrows, int& lo, int& hi) {
  const float u0 = xa - mx, u1 = xb - mx;
  lo = 1;
  hi = 0;
  if (!(u0 <= rx + kCellTol && u1 >= -rx - kCellTol)) return;
  const float s = C01 * inv11;
  const float kk = k2 * inv11;
  const float irx2 = __fdividef(1.0f, rx * rx);
  const float xt = -C01 * inv00 * ry;
  const float xtop = fminf(fmaxf(xt, u0), u1), xbot = fminf(fmaxf(-xt, u0), u1);
  const float ttop = kk * fmaf(-xtop * xtop, irx2, 1.0f), tbot = kk * fmaf(-xbot * xbot, irx2, 1.0f);
  const float htop = ttop > 0.0f ? ttop * rsqrtf(ttop) : 0.0f;
  const float hbot = tbot > 0.0f ? tbot * rsqrtf(tbot) : 0.0f;
  const float ymax = fmaf(-s, xtop, htop), ymin = fmaf(-s, xbot, -hbot);
  // pixel row y has its centres at height y + 0.5
  lo = max(0, __float2int_ru(my + ymin - 0.5f - kCellTol));
  hi = min(nrows - 1, __float2int_rd(my + ymax - 0.5f + kCellTol));
}

// Cells of a TILE x TILE tile (bands of BH pixel rows by columns of 8 pixels)
// whose pixel centres the culling ellipse d^T C d <= k2 touches, as a bit mask:
// band b, column c is bit b * (TILE / 8) + c for 8-row bands (the 8 x 8
// blocks) and 2 (b / 2 * (TILE / 8) + c) + b % 2 for 4-row bands (the 8 x 4
// half-blocks, so the two halves of a block are adjacent bits).  Over a band's
// pixel-centre heights the ellipse spans x in [xmin, xmax]: its chord at height
// dy (from the centre) is centred on -s dy, s = C01 / C00, with half-width
// sqrt((k2 - D dy^2) / C00), D = C11 - C01^2 / C00 = k2 / ry^2 (ry the
// ellipse's half-height), and its right (left) end is furthest out at the
// height dyt of the rightmost point (-dyt), clamped to the band.  A cell is
// touched iff its column's pixel centres meet [xmin, xmax]; the interval is
// widened by 1e-3 pixel so that rounding and the approximate square roots only
// ever add cells (an extra cell adds pixels where every term is below eps).
//   r2 = (C00, C01, C11, rx), r3 = (ry, valid, 1/C00, 1/C11); (mx, my) the
//   tile-relative centre.
template <int TILE, int BH>
__device__ __forceinline__ unsigned ellipse_cells(float4 r2, float4 r3, float mx, float my, float k2) {
  const float ry = r3.x, inv00 = r3.z;
  const float s = r2.y * inv00;
  const float D = k2 / (ry * ry);
  const float dyt = -r2.y * r3.w * r2.w;
  unsigned m = 0u;
#pragma unroll
  for (int b = 0; b < TILE / BH; ++b) {
    const float dya = fmaxf((float)(b * BH) + 0.5f - my, -ry);
    const float dyb = fminf((float)(b * BH + BH) - 0.5f - my, ry);
    if (dya <= dyb) {
      const float dM = fminf(fmaxf(dyt, dya), dyb), dm = fminf(fmaxf(-dyt, dya), dyb);
      const float tM = (k2 - D * dM * dM) * inv00, tm = (k2 - D * dm * dm) * inv00;
      const float xmax = fmaf(-s, dM, mx) + (tM > 0.0f ? tM * rsqrtf(tM) : 0.0f) + kCellTol;
      const float xmin = fmaf(-s, dm, mx) - (tm > 0.0f ? tm * rsqrtf(tm) : 0.0f) - kCellTol;
#pragma unroll
      for (int c = 0; c < TILE / 8; ++c) {
        const int bit = BH == 8 ? b * (TILE / 8) + c : 2 * ((b >> 1) * (TILE / 8) + c) + (b & 1);
        if (xmin <= (float)(8 * c) + 7.5f && xmax >= (float)(8 * c) + 0.5f) m |= 1u << bit;
      }
    }
  }
  return m;
}

// The row units of one (Gaussian, plane, tile): bit c * TILE + y is set when
// the culling ellipse meets the pixel-centre segment of column band c (pixels
// 8c .. 8c + 7) of tile row y.  r0, r2, r3: the Gaussian's record; d its
// offset from the plane; (mx, my) its tile-relative centre on the plane;
// nrows / nbands: the tile's rows and column bands inside the image.  On a
// voxelizer plane the ellipse is the plane's section of the 3D one, d^T C d <=
// k2 - delta^2 / Sigma_zz (its extents scaled to match).
template <int TILE>
__device__ __forceinline__ unsigned row_unit_mask(float4 r0, float4 r2, float4 r3, float d, float mx, float my,
                                                  float k2, bool vox, int nrows, int nbands) {
  float ke = k2, rx = r2.w, ry = r3.x;
  if (vox) {
    ke = k2 - d * d * r0.w;
    if (!(ke > 0.0f)) return 0u;
    const float f = sqrtf(ke / k2);
    rx *= f;
    ry *= f;
  }
  unsigned mask = 0u;
#pragma unroll
  for (int c = 0; c < TILE / 8; ++c) {
    if (c >= nbands) break;
    int lo, hi;
    band_rows(r2.y, r3.z, r3.w, rx, ry, ke, mx, my, (float)(8 * c) + 0.5f, (float)(8 * c) + 7.5f, nrows, lo, hi);
    if (lo <= hi) mask |= ((0xffffffffu >> (31 - (hi - lo))) << lo) << (c * TILE);
  }
  return mask;
}

// The culling cells of one (Gaussian, plane, tile) for the block-culled
// rasterisers: ellipse_cells with, on a voxelizer plane, the plane's section
// of the 3D ellipsoid (k2 - delta^2 / Sigma_zz, extents scaled to match).
template <int TILE, int BH>
__device__ __forceinline__ unsigned plane_cells(float4 r0, float4 r2, float4 r3, float d, float mx, float my,
                                                float k2, bool vox) {
  if (vox) {
    const float k2e = k2 - d * d * r0.w;
    if (!(k2e > 0.0f)) return 0u;
    const float f = sqrtf(k2e / k2);
    return ellipse_cells<TILE, BH>(make_float4(r2.x, r2.y, r2.z, r2.w * f), make_float4(r3.x * f, r3.y, r3.z, r3.w),
                                   mx, my, k2e);
  }
  return ellipse_cells<TILE, BH>(r2, r3, mx, my, k2);
}
// Exponentials 2^(base + B q) of a couple's two pixels (base = A + C q^2): the
// mirrored pixels q and -q of a row share base, so one packed instruction
// finishes each exponent.
// FLOOR = false drops the floor where the caller knows every exponent is above
// kExpUnfloored.
// GRAD selects the backward's exponential (exp2_grad in the polynomial modes).
template <int EXPM, bool FLOOR = true, bool GRAD = false>
__device__ __forceinline__ float2 couple_exp2(float2 B2, float2 q, float2 base) {
  float2 e = __ffma2_rn(B2, q, base);
  if constexpr (FLOOR) {
    e.x = fmaxf(e.x, kExpFloor);
    e.y = fmaxf(e.y, kExpFloor);
  }
  if constexpr (GRAD) return exp2_sel2_grad<EXPM>(e);
  else return exp2_sel2<EXPM>(e);
}

// Exponents at or above this need no floor in exp2_poly (a margin of one over
// kExpFloor covers the rounding between a bound and the exponents it bounds).
// Along a row or over a cell the exponent A + B q + C q^2 (+ row terms) is a
// concave quadratic, so it is smallest at a corner: a unit whose corners are
// all above kExpUnfloored can skip the per-pixel floor.
constexpr float kExpUnfloored = kExpFloor + 1.0f;

// ---------------------------------------------------------------- records
// Per-Gaussian slice-invariant record of the slice renderer (camera frame of the
// slice axis), 64 bytes:
//   r0 = (mu_x, mu_y, mu_z, 1/v)         v = Sigma_zz + sigma_z^2
//   r1 = (a_x, a_y, A, zr)                a = Sigma_{xy,z}/v, A = alpha/sqrt(det Sigma_2d),
//                                         zr = axial half range sqrt(2 v ln(1/eps))
//   r2 = (C00, C01, C11, rx)              C = Sigma_2d^-1, rx = k sqrt(Sigma_2d,xx)
//   r3 = (ry, valid, 1/C00, 1/C11)        reciprocals for the ellipse-tile test
struct __align__(16) SliceRec {
  float4 r0, r1, r2, r3;
};

// ------------------------------------------------------------ rotations
// Rotation matrix of q/|q|, q = (w, x, y, z).
__device__ __forceinline__ void quat_rot(float4 q, float R[3][3], float qn[4], float& qnorm) {
  qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  float inv = 1.0f / qnorm;
  float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  R[0][0] = 1.f - 2.f * (yy + zz); R[0][1] = 2.f * (xy - wz);       R[0][2] = 2.f * (xz + wy);
  R[1][0] = 2.f * (xy + wz);       R[1][1] = 1.f - 2.f * (xx + zz); R[1][2] = 2.f * (yz - wx);
  R[2][0] = 2.f * (xz - wy);       R[2][1] = 2.f * (yz + wx);       R[2][2] = 1.f - 2.f * (xx + yy);
}

// World covariance Sigma = (R D)(R D)^T, D = diag(d); returns the 6 unique entries
// (xx, xy, xz, yy, yz, zz) and M = R D.
__device__ __forceinline__ void covariance(const float R[3][3], const float d[3], float M[3][3],
                                           float S6[6]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * d[c];
  auto dot = [&](int a, int b) { return M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2]; };
  S6[0] = dot(0, 0); S6[1] = dot(0, 1); S6[2] = dot(0, 2);
  S6[3] = dot(1, 1); S6[4] = dot(1, 2); S6[5] = dot(2, 2);
}

// Backward of Sigma = M M^T, M = R diag(dd), dd = mod * s, R = R(q/|q|), given
// the symmetric gradient Gw = dL/dSigma.  Adds dL/ds into gs[3] and writes
// dL/dq (through the normalisation q/|q|) into gq[4].
__device__ __forceinline__ void scale_quat_backward(const float R[3][3], const float M[3][3],
                                                    const float dd[3], const float qn[4], float qnorm,
                                                    float mod, const float Gw[3][3], float gs[3],
                                                    float gq[4]) {
  // dL/dM = 2 Gw M, then M = R D: dL/dR = dL/dM D, dL/dD_c = sum_r R_rc dL/dM_rc
  float gR[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float gm = 2.0f * (Gw[r][0] * M[0][c] + Gw[r][1] * M[1][c] + Gw[r][2] * M[2][c]);
      gR[r][c] = gm * dd[c];
      gs[c] += mod * R[r][c] * gm;
    }
  // dR/d(w, x, y, z) of the unit-quaternion rotation, contracted with gR
  const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  float gw = 2.f * (z * (gR[1][0] - gR[0][1]) + y * (gR[0][2] - gR[2][0]) + x * (gR[2][1] - gR[1][2]));
  float gx = 2.f * (y * (gR[0][1] + gR[1][0]) + z * (gR[0][2] + gR[2][0]) + w * (gR[2][1] - gR[1][2])) -
             4.f * x * (gR[1][1] + gR[2][2]);
  float gy = 2.f * (x * (gR[0][1] + gR[1][0]) + w * (gR[0][2] - gR[2][0]) + z * (gR[1][2] + gR[2][1])) -
             4.f * y * (gR[0][0] + gR[2][2]);
  float gz = 2.f * (w * (gR[1][0] - gR[0][1]) + x * (gR[0][2] + gR[2][0]) + y * (gR[1][2] + gR[2][1])) -
             4.f * z * (gR[0][0] + gR[1][1]);
  // q_n = q / |q|: dL/dq = (g - q_n (q_n . g)) / |q|
  float dot = gw * w + gx * x + gy * y + gz * z;
  float iq = 1.0f / qnorm;
  gq[0] = (gw - w * dot) * iq;
  gq[1] = (gx - x * dot) * iq;
  gq[2] = (gy - y * dot) * iq;
  gq[3] = (gz - z * dot) * iq;
}

// Camera axis permutation: camera coordinate j is world coordinate perm(axis, j).
//   axis 2: (x, y, z); axis 1: (x, z, y); axis 0: (y, z, x).
__host__ __device__ __forceinline__ int axis_perm(int axis, int j) {
  return axis == 2 ? j : (axis == 1 ? (j == 0 ? 0 : (j == 1 ? 2 : 1)) : (j == 0 ? 1 : (j == 1 ? 2 : 0)));
}

__host__ __device__ __forceinline__ int sym_index(int a, int b) {
  // index into (xx, xy, xz, yy, yz, zz)
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// Camera frame of a view [R_c | t] (Sec. S1): mu_c = R_c mu + t, accumulated in
// FP64 and rounded once (the plane positions are compared against it, so an
// oblique view loses no more than the rounding of mu_c itself), and the unique
// entries (xx, xy, xz, yy, yz, zz) of Sigma_c = R_c Sigma R_c^T.  For a
// permutation R_c both are exact.
__device__ __forceinline__ void camera_frame(const float* __restrict__ Rc, const float* __restrict__ tc,
                                             const float* __restrict__ mu, const float Sw[6], float muc[3],
                                             float Sc[6]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double acc = (double)tc[r];
    acc = fma((double)Rc[3 * r], (double)mu[0], acc);
    acc = fma((double)Rc[3 * r + 1], (double)mu[1], acc);
    acc = fma((double)Rc[3 * r + 2], (double)mu[2], acc);
    muc[r] = (float)acc;
  }
  float T[3][3];  // R_c Sigma
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      T[u][k] = fmaf(Rc[3 * u + 2], Sw[sym_index(2, k)],
                     fmaf(Rc[3 * u + 1], Sw[sym_index(1, k)], Rc[3 * u] * Sw[sym_index(0, k)]));
  auto sc = [&](int u, int w) {
    return fmaf(T[u][2], Rc[3 * w + 2], fmaf(T[u][1], Rc[3 * w + 1], T[u][0] * Rc[3 * w]));
  };
  Sc[0] = sc(0, 0); Sc[1] = sc(0, 1); Sc[2] = sc(0, 2);
  Sc[3] = sc(1, 1); Sc[4] = sc(1, 2); Sc[5] = sc(2, 2);
}

// --------------------------------------------------- ellipse vs rectangle
// Minimum over the rectangle [x0, x1] x [y0, y1] of q(p) = (p-m)^T C (p-m),
// C = [[c00, c01], [c01, c11]] positive definite, compared with k2.  Written with
// explicit rounding intrinsics so that the pair count and the pair emission (two
// kernels) take bit-identical decisions.
__device__ __forceinline__ float qform(float c00, float c01, float c11, float dx, float dy) {
  float t = __fmaf_rn(c01, __fmul_rn(2.0f, dy), __fmul_rn(c00, dx));
  return __fmaf_rn(t, dx, __fmul_rn(__fmul_rn(c11, dy), dy));
}

// Minimum of q along one edge: the fixed coordinate offset is dfix, the free one
// runs over [dlo, dhi]; the free-coordinate minimiser is -c01 dfix / c_var
// (inv_var = 1 / c_var is precomputed per Gaussian).
__device__ __forceinline__ float edge_min(float c_fixed, float c01, float c_var, float inv_var, float dfix,
                                          float dlo, float dhi, bool fixed_is_x) {
  float dstar = __fmul_rn(-__fmul_rn(c01, dfix), inv_var);
  dstar = fminf(fmaxf(dstar, dlo), dhi);
  return fixed_is_x ? qform(c_fixed, c01, c_var, dfix, dstar) : qform(c_var, c01, c_fixed, dstar, dfix);
}

__device__ __forceinline__ bool ellipse_hits_rect(float mx, float my, float c00, float c01, float c11,
                                                  float inv00, float inv11, float k2, float x0, float x1,
                                                  float y0, float y1) {
  if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
  float dxl = __fsub_rn(x0, mx), dxh = __fsub_rn(x1, mx);
  float dyl = __fsub_rn(y0, my), dyh = __fsub_rn(y1, my);
  float m = edge_min(c00, c01, c11, inv11, dxl, dyl, dyh, true);
  m = fminf(m, edge_min(c00, c01, c11, inv11, dxh, dyl, dyh, true));
  m = fminf(m, edge_min(c11, c01, c00, inv00, dyl, dxl, dxh, false));
  m = fminf(m, edge_min(c11, c01, c00, inv00, dyh, dxl, dxh, false));
  return m <= k2;
}

// ------------------------------------------------------------ misc
__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace gp
