// codec.cu -- the Gaussian-set codec of the paper's storage path (Sec. 4,
// "Quantization and compression"), sm_103a: Morton (Z-order) sort, quantisation
// (positions to the bounding box at B bits per axis, log scales, intensities
// and half-sphere quaternion components at 12 bits), per-attribute delta
// streams; the LZMA stage stays on the host.
//
// Encode (one call, synchronous for the bounding-box readback):
//   K-minmax     bounding box of the positions, range of the scales, argument
//                check (two-stage block reduction, no float atomics)
//   K-quant      per Gaussian: 11 codes and the 3B-bit Morton key (lo / hi words)
//   sort         stable LSD radix sort on the key: low word, then the high word
//                of the low-word order (the library's radix sort, two calls)
//   K-delta      codes gathered in Morton order, differenced, zigzag-mapped
// Decode:
//   K-unzig      zigzag -> two's-complement deltas (uint32)
//   scan         one exclusive scan over the 11 concatenated streams (mod 2^32;
//                each stream subtracts its starting carry)
//   K-dequant    codes -> fp32 parameters
//
// Every integer decision is taken with separately rounded fp32 operations
// (__fsub_rn / __fmul_rn / __fadd_rn / __fdiv_rn / __fsqrt_rn: no contraction),
// except the scale code, which counts the double-precision thresholds
// exp(L0 + (k - 1/2) D), k = 1..4095, not above the scale (round to nearest in
// the log domain without a device logarithm).  The device compares the fp32
// scale with each threshold's ceiling in fp32 (the smallest float not below
// it), which takes exactly the double comparison's decision for every fp32
// scale.  The 11 codes of a Gaussian are kept together (32 bytes) so that the
// Morton-order gather reads two 16-byte vectors per Gaussian; decoded scales
// come from a 4096-entry table of exp(L0 + c D) computed in double on the
// device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gp_internal.h"

namespace gp {

namespace {

constexpr int kThreads = 256;
constexpr int kScaleLevels = 4095;  // 12-bit codes 0..4095

constexpr int kCodeStride = 16;      // uint16 slots per Gaussian in the code buffer (11 used)

struct QuantArgs {
  float lo[3], inv[3];
  int top;          // 2^B - 1
  int bits;
  int scale_range;  // 0: all scales equal (codes 0)
  const float* th;  // kScaleLevels thresholds, each rounded up to fp32
};

struct DequantArgs {
  float lo[3], step[3];
  const float* scale_of;  // decoded scale of each 12-bit code
};

__device__ __forceinline__ void mm_merge(float* a, const float* b) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[2 * k] = fminf(a[2 * k], b[2 * k]);
    a[2 * k + 1] = fmaxf(a[2 * k + 1], b[2 * k + 1]);
  }
}

// per block: (min, max) of mu x, y, z and of all scales; count of invalid Gaussians
__global__ void __launch_bounds__(kThreads) k_codec_minmax(const float* __restrict__ mu,
                                                          const float* __restrict__ scale,
                                                          const float* __restrict__ quat,
                                                          const float* __restrict__ alpha, int64_t n,
                                                          float* __restrict__ part, unsigned* __restrict__ bad) {
  float m[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    m[2 * k] = INFINITY;
    m[2 * k + 1] = -INFINITY;
  }
  unsigned nbad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    bool ok = isfinite(alpha[i]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float x = mu[3 * i + k], s = scale[3 * i + k];
      ok = ok && isfinite(x) && isfinite(s) && s > 0.0f;
      m[2 * k] = fminf(m[2 * k], x);
      m[2 * k + 1] = fmaxf(m[2 * k + 1], x);
      m[6] = fminf(m[6], s);
      m[7] = fmaxf(m[7], s);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) ok = ok && isfinite(quat[4 * i + k]);
    nbad += ok ? 0u : 1u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float v = __shfl_xor_sync(0xffffffffu, m[k], o);
      m[k] = (k & 1) ? fmaxf(m[k], v) : fminf(m[k], v);
    }
    nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
  }
  __shared__ float sm[kThreads / 32][8];
  __shared__ unsigned sb[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sm[threadIdx.x >> 5][k] = m[k];
    sb[threadIdx.x >> 5] = nbad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) {
      mm_merge(sm[0], sm[w]);
      sb[0] += sb[w];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[8 * blockIdx.x + k] = sm[0][k];
    atomicAdd(bad, sb[0]);
  }
}

// the blocks' partials merged by one block (min and max are exact, so the
// order of the merge does not matter)
__global__ void __launch_bounds__(kThreads) k_codec_minmax_final(const float* __restrict__ part, int nb,
                                                                float* __restrict__ out) {
  float m[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    m[2 * k] = INFINITY;
    m[2 * k + 1] = -INFINITY;
  }
  for (int b = threadIdx.x; b < nb; b += kThreads) mm_merge(m, part + 8 * b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float v = __shfl_xor_sync(0xffffffffu, m[k], o);
      m[k] = (k & 1) ? fmaxf(m[k], v) : fminf(m[k], v);
    }
  }
  __shared__ float sm[kThreads / 32][8];
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sm[threadIdx.x >> 5][k] = m[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) mm_merge(sm[0], sm[w]);
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = sm[0][k];
  }
}

__device__ __forceinline__ int q_affine(float v, float lo, float inv, int top) {
  if (!(inv > 0.0f)) return 0;
  const float t = __fadd_rn(__fmul_rn(__fsub_rn(v, lo), inv), 0.5f);
  const float f = floorf(t);
  return f < 0.0f ? 0 : (f > (float)top ? top : (int)f);
}

__device__ __forceinline__ int q_12(float t_before_half) {
  const float f = floorf(__fadd_rn(t_before_half, 0.5f));
  return f < 0.0f ? 0 : (f > 4095.0f ? 4095 : (int)f);
}

__global__ void __launch_bounds__(kThreads) k_codec_quant(QuantArgs p, const float* __restrict__ mu,
                                                         const float* __restrict__ scale,
                                                         const float* __restrict__ quat,
                                                         const float* __restrict__ alpha, int64_t n,
                                                         uint16_t* __restrict__ codes, uint32_t* __restrict__ klo,
                                                         uint32_t* __restrict__ khi) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  uint32_t cw[kCodeStride / 2] = {};  // the Gaussian's codes, two per word (code 2m in the low half)
  int pc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) pc[k] = q_affine(mu[3 * i + k], p.lo[k], p.inv[k], p.top);
  unsigned long long key = 0;
  for (int j = 0; j < p.bits; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) key |= (unsigned long long)((pc[a] >> j) & 1) << (3 * j + a);
  klo[i] = (uint32_t)key;
  khi[i] = (uint32_t)(key >> 32);
  int c11[11];
#pragma unroll
  for (int k = 0; k < 3; ++k) c11[k] = pc[k];
  // scales: number of thresholds not above s
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int c = 0;
    if (p.scale_range) {
      const float sv = scale[3 * i + k];
      int lo = 0, hi = kScaleLevels;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (p.th[mid] <= sv) lo = mid + 1;
        else hi = mid;
      }
      c = lo;
    }
    c11[3 + k] = c;
  }
  // quaternion: normalised (w, x, y, z summed in order), folded to w >= 0
  const float4 q = reinterpret_cast<const float4*>(quat)[i];
  float n2 = __fmul_rn(q.x, q.x);
  n2 = __fadd_rn(n2, __fmul_rn(q.y, q.y));
  n2 = __fadd_rn(n2, __fmul_rn(q.z, q.z));
  n2 = __fadd_rn(n2, __fmul_rn(q.w, q.w));
  const float nrm = __fsqrt_rn(n2);
  float c4[4] = {0.f, 0.f, 0.f, 0.f};
  if (nrm > 0.0f) {
    c4[0] = __fdiv_rn(q.x, nrm);
    c4[1] = __fdiv_rn(q.y, nrm);
    c4[2] = __fdiv_rn(q.z, nrm);
    c4[3] = __fdiv_rn(q.w, nrm);
  }
  if (c4[0] < 0.0f) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c4[k] = -c4[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) c11[6 + k] = q_12(__fmul_rn(__fadd_rn(c4[k], 1.0f), 2047.5f));
  const float a = fminf(fmaxf(alpha[i], 0.0f), 1.0f);
  c11[10] = q_12(__fmul_rn(a, 4095.0f));
#pragma unroll
  for (int k = 0; k < 11; ++k) cw[k >> 1] |= (uint32_t)(uint16_t)c11[k] << (16 * (k & 1));
  uint4* dst = reinterpret_cast<uint4*>(codes + (size_t)i * kCodeStride);
  dst[0] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
  dst[1] = make_uint4(cw[4], cw[5], cw[6], cw[7]);
}

__global__ void k_codec_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                                   uint32_t* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__device__ __forceinline__ void load_codes(const uint16_t* __restrict__ codes, uint32_t g, uint32_t* w) {
  const uint4* src = reinterpret_cast<const uint4*>(codes + (size_t)g * kCodeStride);
  const uint4 a = src[0], b = src[1];
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

__global__ void __launch_bounds__(kThreads) k_codec_delta(const uint16_t* __restrict__ codes,
                                                         const uint32_t* __restrict__ order, int64_t n,
                                                         uint16_t* __restrict__ streams,
                                                         uint32_t* __restrict__ order_out) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const uint32_t cur = order[i];
  uint32_t wc[8], wp[8] = {};
  load_codes(codes, cur, wc);
  if (i > 0) load_codes(codes, order[i - 1], wp);
#pragma unroll
  for (int a = 0; a < 11; ++a) {
    const int c = (int)((wc[a >> 1] >> (16 * (a & 1))) & 0xffffu);
    const int b = (int)((wp[a >> 1] >> (16 * (a & 1))) & 0xffffu);
    const int d = c - b;
    streams[(int64_t)a * n + i] = (uint16_t)(d >= 0 ? 2 * d : -2 * d - 1);
  }
  if (order_out) order_out[i] = cur;
}

// decoded scale of every 12-bit code: exp(L0 + c D) in double, rounded to fp32
__global__ void k_codec_scale_table(double L0, double D, float* __restrict__ table) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c <= kScaleLevels) table[c] = (float)exp(L0 + (double)c * D);
}

__global__ void __launch_bounds__(kThreads) k_codec_unzig(const uint16_t* __restrict__ streams, int64_t total,
                                                         uint32_t* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= total) return;
  const int z = streams[i];
  const int v = (z & 1) ? -((z + 1) >> 1) : (z >> 1);
  d[i] = (uint32_t)v;
}

__global__ void __launch_bounds__(kThreads) k_codec_dequant(DequantArgs p, const uint32_t* __restrict__ d,
                                                           const uint32_t* __restrict__ ex, int64_t n,
                                                           float* __restrict__ mu, float* __restrict__ scale,
                                                           float* __restrict__ quat, float* __restrict__ alpha) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  int c[11];
#pragma unroll
  for (int a = 0; a < 11; ++a) {
    const int64_t o = (int64_t)a * n;
    c[a] = (int)(ex[o + i] + d[o + i] - ex[o]);  // inclusive prefix of stream a, mod 2^32
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) mu[3 * i + k] = __fadd_rn(p.lo[k], __fmul_rn((float)c[k], p.step[k]));
#pragma unroll
  for (int k = 0; k < 3; ++k) scale[3 * i + k] = p.scale_of[min(max(c[3 + k], 0), kScaleLevels)];
  float4 q;
  q.x = __fsub_rn(__fdiv_rn((float)c[6], 2047.5f), 1.0f);
  q.y = __fsub_rn(__fdiv_rn((float)c[7], 2047.5f), 1.0f);
  q.z = __fsub_rn(__fdiv_rn((float)c[8], 2047.5f), 1.0f);
  q.w = __fsub_rn(__fdiv_rn((float)c[9], 2047.5f), 1.0f);
  reinterpret_cast<float4*>(quat)[i] = q;
  alpha[i] = __fdiv_rn((float)c[10], 4095.0f);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

#define CODEC_TRY(x)             \
  do {                           \
    const gp_status s_ = (x);    \
    if (s_ != GP_OK) return s_;  \
  } while (0)

}  // namespace

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_encode(gp_ctx* ctx, const gp_set* set, int pos_bits, gp_codec_header* header, uint16_t* streams,
                    uint32_t* order, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!set || !header || set->n < 0) return set_err(c, GP_ERR_ARG, "NULL set / header or negative n");
  if (pos_bits < 1 || pos_bits > 15) return set_err(c, GP_ERR_ARG, "pos_bits must be in 1..15");
  if (set->n > (int64_t)UINT32_MAX / 2) return set_err(c, GP_ERR_ARG, "too many Gaussians for one stream set");
  const int64_t n = set->n;
  memset(header, 0, sizeof(*header));
  header->n = n;
  header->pos_bits = pos_bits;
  if (n == 0) return GP_OK;
  if (!set->mu || !set->scale || !set->quat || !set->alpha || !streams)
    return set_err(c, GP_ERR_ARG, "NULL pointer");
  if ((uintptr_t)set->quat & 15u) return set_err(c, GP_ERR_ARG, "quat must be 16-byte aligned");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  c->bin_key.valid = false;  // the workspace's pair buffers are reused below
  const int nb = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * (int64_t)c->sm_count);
  // scratch: codes | klo | khi | vals (4 buffers) | gather | th | part | mm | bad | n_dev
  const size_t o_codes = 0;
  const size_t o_klo = o_codes + align256((size_t)kCodeStride * n * 2);
  const size_t o_khi = o_klo + align256((size_t)n * 4);
  const size_t o_k2 = o_khi + align256((size_t)n * 4);
  const size_t o_v1 = o_k2 + align256((size_t)n * 4);
  const size_t o_v2 = o_v1 + align256((size_t)n * 4);
  const size_t o_g = o_v2 + align256((size_t)n * 4);
  const size_t o_th = o_g + align256((size_t)n * 4);
  const size_t o_part = o_th + align256((size_t)kScaleLevels * 4);
  const size_t o_mm = o_part + align256((size_t)nb * 32);
  const size_t o_nd = o_mm + 256;
  const size_t total = o_nd + 256;
  BinBufs& b = c->b;
  CODEC_TRY(ws_reserve(c, b.codec, total));
  CODEC_TRY(ws_reserve(c, b.sort_tmp, (size_t)radix_temp_bytes(n)));
  char* base = (char*)b.codec.ptr;
  uint16_t* codes = (uint16_t*)(base + o_codes);
  uint32_t* klo = (uint32_t*)(base + o_klo);
  uint32_t* khi = (uint32_t*)(base + o_khi);
  uint32_t* k2 = (uint32_t*)(base + o_k2);
  uint32_t* v1 = (uint32_t*)(base + o_v1);
  uint32_t* v2 = (uint32_t*)(base + o_v2);
  uint32_t* g = (uint32_t*)(base + o_g);
  float* th = (float*)(base + o_th);
  float* part = (float*)(base + o_part);
  float* mm = (float*)(base + o_mm);
  unsigned* bad = (unsigned*)(base + o_mm + 32);  // read back with the 8 floats before it
  unsigned long long* n_dev = (unsigned long long*)(base + o_nd);
  // bounding box, scale range, argument check
  if (cudaMemsetAsync(bad, 0, 4, st) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "codec memset");
  k_codec_minmax<<<nb, kThreads, 0, st>>>(set->mu, set->scale, set->quat, set->alpha, n, part, bad);
  k_codec_minmax_final<<<1, kThreads, 0, st>>>(part, nb, mm);
  note_launch(2);
  float h[9];
  if (cudaMemcpyAsync(h, mm, 36, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_err(c, cudaGetLastError(), "codec bounding box");
  unsigned hbad;
  memcpy(&hbad, &h[8], 4);
  if (hbad) return set_err(c, GP_ERR_ARG, "non-finite parameter or scale <= 0");
  QuantArgs qa;
  const int top = (1 << pos_bits) - 1;
  for (int k = 0; k < 3; ++k) {
    header->lo[k] = h[2 * k];
    header->hi[k] = h[2 * k + 1];
    const float d = h[2 * k + 1] - h[2 * k];  // rounded once, as the decoder's step uses it
    qa.lo[k] = h[2 * k];
    qa.inv[k] = d > 0.0f ? (float)top / d : 0.0f;
  }
  header->log_s_min = log((double)h[6]);
  header->log_s_max = log((double)h[7]);
  qa.top = top;
  qa.bits = pos_bits;
  qa.scale_range = header->log_s_max > header->log_s_min ? 1 : 0;
  qa.th = th;
  if (qa.scale_range) {
    // each threshold's fp32 ceiling: for an fp32 scale s, t <= (double)s exactly
    // when ceil32(t) <= s
    std::vector<float> t(kScaleLevels);
    const double D = (header->log_s_max - header->log_s_min) / (double)kScaleLevels;
    for (int k = 1; k <= kScaleLevels; ++k) {
      const double tk = exp(header->log_s_min + ((double)k - 0.5) * D);
      float f = (float)tk;
      if ((double)f < tk) f = nextafterf(f, INFINITY);
      t[k - 1] = f;
    }
    if (cudaMemcpyAsync(th, t.data(), t.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return cuda_err(c, cudaGetLastError(), "codec thresholds");
  }
  const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
  k_codec_quant<<<grid, kThreads, 0, st>>>(qa, set->mu, set->scale, set->quat, set->alpha, n, codes, klo, khi);
  note_launch();
  // stable order by the 3B-bit key: low word, then high word of that order
  const unsigned long long nn = (unsigned long long)n;
  if (cudaMemcpyAsync(n_dev, &nn, 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return cuda_err(c, cudaGetLastError(), "codec count");
  const int kb = 3 * pos_bits;
  bool alt = false;
  cudaError_t e = radix_sort_pairs(klo, v1, k2, v2, n_dev, (uint32_t)n, std::min(kb, 32), b.sort_tmp.ptr, st, &alt);
  if (e != cudaSuccess) return cuda_err(c, e, "codec sort");
  uint32_t* perm = alt ? v2 : v1;
  if (kb > 32) {
    k_codec_gather_u32<<<grid, kThreads, 0, st>>>(khi, perm, n, g);  // high words in low-word order
    note_launch();
    uint32_t* perm1 = perm == v1 ? v1 : v2;
    uint32_t* spare = perm == v1 ? v2 : v1;
    // sort the high words (identity values), then compose with the first order
    cudaMemcpyAsync(spare, perm1, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    bool alt2 = false;
    e = radix_sort_pairs(g, perm1, khi, klo, n_dev, (uint32_t)n, kb - 32, b.sort_tmp.ptr, st, &alt2);
    if (e != cudaSuccess) return cuda_err(c, e, "codec sort");
    uint32_t* perm2 = alt2 ? klo : perm1;
    k_codec_gather_u32<<<grid, kThreads, 0, st>>>(spare, perm2, n, g);
    note_launch();
    perm = g;
  }
  k_codec_delta<<<grid, kThreads, 0, st>>>(codes, perm, n, streams, order);
  note_launch();
  return cuda_err(c, cudaGetLastError(), "codec encode");
}

gp_status gp_decode(gp_ctx* ctx, const gp_codec_header* header, const uint16_t* streams, float* mu, float* scale,
                    float* quat, float* alpha, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!header || header->n < 0 || header->pos_bits < 1 || header->pos_bits > 15)
    return set_err(c, GP_ERR_ARG, "bad codec header");
  const int64_t n = header->n;
  if (n == 0) return GP_OK;
  if (!streams || !mu || !scale || !quat || !alpha) return set_err(c, GP_ERR_ARG, "NULL pointer");
  if ((uintptr_t)quat & 15u) return set_err(c, GP_ERR_ARG, "quat must be 16-byte aligned");
  if (!isfinite(header->log_s_min) || !isfinite(header->log_s_max) || header->log_s_max < header->log_s_min)
    return set_err(c, GP_ERR_ARG, "bad scale range in the header");
  for (int k = 0; k < 3; ++k)
    if (!isfinite(header->lo[k]) || !isfinite(header->hi[k]) || header->hi[k] < header->lo[k])
      return set_err(c, GP_ERR_ARG, "bad bounding box in the header");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t tot = 11 * n;
  BinBufs& b = c->b;
  CODEC_TRY(ws_reserve(c, b.codec, 2 * align256((size_t)tot * 4) + align256((kScaleLevels + 1) * 4)));
  CODEC_TRY(ws_reserve(c, b.scan_tmp, (size_t)scan_temp_bytes(tot)));
  uint32_t* d = (uint32_t*)b.codec.ptr;
  uint32_t* ex = (uint32_t*)((char*)b.codec.ptr + align256((size_t)tot * 4));
  float* scale_of = (float*)((char*)b.codec.ptr + 2 * align256((size_t)tot * 4));
  k_codec_scale_table<<<(kScaleLevels + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
      header->log_s_min, (header->log_s_max - header->log_s_min) / (double)kScaleLevels, scale_of);
  note_launch();
  k_codec_unzig<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, st>>>(streams, tot, d);
  note_launch();
  cudaError_t e = exclusive_scan<uint32_t>(d, ex, tot, nullptr, b.scan_tmp.ptr, st);
  if (e != cudaSuccess) return cuda_err(c, e, "codec scan");
  DequantArgs p;
  const float top = (float)((1 << header->pos_bits) - 1);
  for (int k = 0; k < 3; ++k) {
    p.lo[k] = header->lo[k];
    p.step[k] = (header->hi[k] - header->lo[k]) / top;
  }
  p.scale_of = scale_of;
  k_codec_dequant<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(p, d, ex, n, mu, scale, quat,
                                                                                   alpha);
  note_launch();
  return cuda_err(c, cudaGetLastError(), "codec decode");
}

}  // extern "C"
