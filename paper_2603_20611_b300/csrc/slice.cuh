// slice.cuh -- launch interface of the slice-renderer kernels (slice.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_common.cuh"

namespace gp {

// Arguments shared by every slice-renderer kernel.
struct SliceArgs {
  const float* mu;
  const float* scale;
  const float* quat;
  const float* alpha;
  int n;
  float mod;
  float Rc[9];    // view [R_c | t]: camera coordinates x_c = R_c x + t (row-major R_c)
  float tc[3];
  float sigma2;   // sigma_z^2
  float k2;       // 2 ln(1/eps): squared Mahalanobis culling radius
  int vox;        // 1: voxelizer planes (Eq. 12): sigma_z = 0 and amplitude alpha, not alpha/sqrt(det Sigma_2d)
  const float* zs;      // [S] plane positions sorted ascending
  const int* zorder;    // [S] slice index of sorted position j
  const float* zorig;   // [S] plane position of slice index s
  int S, H, W;
  int tile, TX, TY;     // tile side and tile grid (TX * TY tiles per slice)
  // batched launches: this item's first Gaussian and first (slice, tile) key in
  // the batch-wide index spaces (0 for a single render), its output image,
  // upstream gradient and parameter-gradient outputs
  int gbase;
  uint32_t key_base;
  float* out;
  const float* dL_dI;
  float *d_mu, *d_scale, *d_quat, *d_alpha;
};

// Items of a batched launch, in device memory: args[k] describes item k, whose
// Gaussians are [gstart[k], gstart[k+1]) and keys [kstart[k], kstart[k+1]).
struct BatchItems {
  const SliceArgs* args;
  const int* gstart;
  const uint32_t* kstart;
  int n_items;
  int n_gauss;        // gstart[n_items]
  uint32_t n_keys;    // kstart[n_items]
};

void launch_slice_pre_batch(const BatchItems& b, SliceRec* rec, unsigned long long* counts, unsigned long long* wsum,
                            cudaStream_t st);
void launch_slice_emit_batch(const BatchItems& b, const SliceRec* rec, const unsigned long long* woff,
                             const unsigned long long* counts, unsigned long long* offsets, uint32_t cap,
                             uint32_t* keys, uint32_t* emit_gid, cudaStream_t st);
void launch_slice_bwd_pre_batch(const BatchItems& b, const float* accum, cudaStream_t st);
void launch_det_reduce_n(int n, const unsigned long long* offsets, const unsigned long long* counts,
                         const float4* partial, float* accum, unsigned long long cap, cudaStream_t st);
// Persistent block-culled rasterisers over every (item, slice, tile) key of a
// batch: CTAs take chunks of keys from *work (zeroed before each launch).
cudaError_t launch_raster_fwd_batch(const BatchItems& b, bool rows, int tile, int chunk, int ctas, int exp_mode,
                                    const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                    const uint2* ranges, unsigned* work, cudaStream_t st);
cudaError_t launch_raster_bwd_batch(const BatchItems& b, bool rows, int tile, int chunk, int ctas, int exp_mode, bool det,
                                    const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                    const uint2* ranges, float* accum, float4* partial, unsigned* work,
                                    cudaStream_t st);
int raster_batch_ctas_per_sm(bool rows, int tile, int chunk, bool backward, int exp_mode);

// The item of batch key x: the last k with t[k] <= x (t ascending, t[0] = 0).
template <typename T>
__device__ __forceinline__ int find_item_k(const T* __restrict__ t, int n, T x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (t[m] <= x) lo = m; else hi = m;
  }
  return lo;
}

// Per-thread rasterisers over every (item, slice, tile) key of a batch (one
// CTA per key): px pixels per thread, as gp_config.fwd_px / bwd_px.
cudaError_t launch_raster_fwd_px_batch(const BatchItems& b, int tile, int px, int exp_mode, const SliceRec* rec,
                                       const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                       cudaStream_t st);
cudaError_t launch_raster_bwd_px_batch(const BatchItems& b, int tile, int px, int exp_mode, bool det,
                                       const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                                       const uint2* ranges, float* accum, float4* partial, cudaStream_t st);

// K-pre: records, per-Gaussian pair counts and per-warp (32 Gaussians) totals.
void launch_slice_pre(const SliceArgs& a, SliceRec* rec, unsigned long long* counts, unsigned long long* wsum,
                      cudaStream_t st);
// K-emit: (slice, tile) keys and Gaussian ids, placed by woff (the exclusive
// scan of K-pre's per-warp totals); writes each Gaussian's offset into offsets;
// no pair at or past index cap is written.
void launch_slice_emit(const SliceArgs& a, const SliceRec* rec, const unsigned long long* woff,
                       const unsigned long long* counts, unsigned long long* offsets, uint32_t* keys,
                       uint32_t* emit_gid, cudaStream_t st, unsigned long long cap = ~0ull);
// K-range: [start, end) of each key in the sorted key list; ranges must be zeroed.
void launch_ranges(const uint32_t* keys, const unsigned long long* n_dev, uint32_t cap, uint32_t nkeys,
                   uint2* ranges, cudaStream_t st);
// K-fwd.
// pairs: the binned (Gaussian, slice, tile) pairs, which choose the occupancy
// of the default forward (see launch_raster_fwd_blocked).
// px > 0: the per-thread kernel; px = 0: the default kernels of form `raster`
// (GP_RASTER_*).
cudaError_t launch_raster_fwd(const SliceArgs& a, int px, int raster, int exp_mode, const SliceRec* rec,
                              const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                              float* out, cudaStream_t st, uint32_t pairs);
// K-bwd-raster; atomic mode adds into accum [n][10] (zeroed), deterministic mode
// writes per-pair partials [pairs][8].
cudaError_t launch_raster_bwd(const SliceArgs& a, int px, int raster, int exp_mode, bool deterministic,
                              const SliceRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                              const uint2* ranges, const float* dL_dI, float* accum, float4* partial,
                              cudaStream_t st);
// K-bwd-pre: accumulators -> parameter gradients.
void launch_slice_bwd_pre(const SliceArgs& a, const float* accum, float* d_mu, float* d_scale,
                          float* d_quat, float* d_alpha, cudaStream_t st);
// K-loss.
void launch_mse(const float* I, const float* T, const int* t_index, int S, int64_t HW, float* dL_dI,
                float* loss, float* tmp, cudaStream_t st);
int mse_tmp_floats(int S, int64_t HW);
// Algorithmic evaluation count (pixels inside the culling ellipse), added into *out.
void launch_count_evals(const SliceArgs& a, const SliceRec* rec, unsigned long long* out,
                        cudaStream_t st);
// Pixels the default rasterisers of the given form evaluate, added into out[0]
// (forward) and out[1] (backward).
void launch_count_units(const SliceArgs& a, const SliceRec* rec, bool rows_f, bool rows_b, unsigned long long* out,
                        cudaStream_t st);
void launch_exp2_eval(const float* x, float* y, int64_t n, int mode, cudaStream_t st);

// Block-culled rasterisers (raster.cu), the default for 16 x 16 tiles.  The
// forward runs at 8 CTAs per SM (more registers, more exponentials in flight)
// when the tiles hold kDenseTilePairs or more pairs on average, else at 12
// (sparse tiles, as on voxelizer planes, are latency-bound).
constexpr uint32_t kDenseTilePairs = 48;
// Row units when raster is GP_RASTER_ROWS, or GP_RASTER_AUTO for the forward
// and for the backward on voxelizer planes (a.vox), with a per-pixel
// exponential; block-culled otherwise.
bool raster_rows_form(const SliceArgs& a, int raster, int exp_mode, bool backward);
cudaError_t launch_raster_fwd_blocked(const SliceArgs& a, int raster, int exp_mode, const SliceRec* rec, const uint32_t* vals,
                                      const uint32_t* emit_gid, const uint2* ranges, float* out, cudaStream_t st,
                                      uint32_t pairs);
cudaError_t launch_raster_bwd_blocked(const SliceArgs& a, int raster, int exp_mode, bool det, const SliceRec* rec,
                                      const uint32_t* vals, const uint32_t* emit_gid, const uint2* ranges,
                                      const float* dL_dI, float* accum, float4* partial, cudaStream_t st);

// Supported pixels-per-thread of the rasterisers for a tile side (0 = the
// default: block-culled kernel for 16 x 16 tiles, one pixel per thread for 8 x 8).
bool fwd_px_supported(int tile, int px);
bool bwd_px_supported(int tile, int px);

}  // namespace gp
