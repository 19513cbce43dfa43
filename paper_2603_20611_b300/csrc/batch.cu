// batch.cu -- batched slice rendering: many Gaussian sets of uneven sizes, each
// with its own slice stack, image size, sigma_z and slice axis, rendered (and
// differentiated) by one graph launch.
//
// The plan concatenates the items into batch-wide index spaces -- Gaussians
// [gstart[k], gstart[k+1]) and (slice, tile) keys [kstart[k], kstart[k+1]) for
// item k -- so a single K-pre, scan, K-emit, radix sort and K-range bin every
// item at once, and persistent rasterisers take (item, slice, tile) keys from a
// global work counter, which balances items of very different sizes.  The
// sequence (memsets, binning, forward, per-item MSE, backward, gradient finish,
// overflow check) is captured once into a CUDA graph; gp_batch_run replays it.
// Pair buffers are sized at plan time from a real count plus headroom; a run
// whose pairs exceed them clamps every kernel to the capacity (no access out of
// bounds) and raises a flag that gp_batch_wait reports as GP_ERR_OVERFLOW.
//
// The autotuner (GP_BATCH_AUTOTUNE) times the plan's own workload for each tile
// side (8, 16) and, for the forward and the backward separately, each
// rasteriser form: block-culled (four warps per tile, 8 x 8 / 8 x 4 cells) at
// each staging chunk (forward 64/128/256, backward 32/64/128 Gaussians per
// round); row units (one warp per tile, 8-pixel row segments); and one thread
// per pixel group at each number of pixels per thread (forward 1/2/4,
// backward 2/4/8 on 16 x 16 tiles; 1/2 and 2 on 8 x 8), and keeps the fastest
// combination.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

__global__ void k_overflow_flag(const unsigned long long* __restrict__ total, unsigned long long cap,
                                unsigned* __restrict__ flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *flag = (*total > cap) ? 1u : 0u;
}

}  // namespace gp

using namespace gp;

struct gp_plan {
  Ctx* c = nullptr;
  std::vector<gp_batch_item> items;
  std::vector<View> views;  // per item, copied at plan time (item.view is not kept)
  int flags = 0;
  int tile = 16, fchunk = 128, bchunk = 64, ctas_f = 0, ctas_b = 0;
  // forward / backward rasteriser form (GP_RASTER_BLOCK, _ROWS or _PIXELS) and, for the per-thread
  // form, pixels per thread
  int fform = GP_RASTER_BLOCK, bform = GP_RASTER_BLOCK, fpx = 0, bpx = 0;
  bool any_fwd = false, any_bwd = false, det = false;
  int n_gauss = 0;
  uint32_t n_keys = 0;
  uint32_t cap = 0;
  int64_t bytes = 0;
  std::vector<SliceArgs> args;
  std::vector<int> gstart;
  std::vector<uint32_t> kstart;
  std::vector<int64_t> img_off;  // offsets of the plan-owned images / gradients per item (floats)
  // device memory owned by the plan
  std::vector<void*> allocs;
  SliceArgs* d_args = nullptr;
  int* d_gstart = nullptr;
  uint32_t* d_kstart = nullptr;
  float* d_z = nullptr;  // per item: sorted positions, order (as int), positions by index
  SliceRec* rec = nullptr;
  unsigned long long *counts = nullptr, *offsets = nullptr, *total = nullptr;
  unsigned long long *wsum = nullptr, *woff = nullptr;  // per warp of 32 Gaussians: pair total, its scan
  uint32_t *keys = nullptr, *vals = nullptr, *keys_alt = nullptr, *vals_alt = nullptr, *emit_gid = nullptr;
  const uint32_t *sk = nullptr, *sv = nullptr;  // sorted keys / values (one of the two ping-pong buffers)
  uint2* ranges = nullptr;
  void *scan_tmp = nullptr, *sort_tmp = nullptr, *mse_tmp = nullptr;
  float* accum = nullptr;
  float4* partial = nullptr;
  float* images = nullptr;  // plan-owned forward images (items with a target but no out)
  float* grads_in = nullptr;  // plan-owned dL/dI of items with a target
  unsigned* work = nullptr;  // two work counters
  unsigned* flag = nullptr;
  unsigned* h_flag = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace gp {

static gp_status plan_alloc(gp_plan* p, void** ptr, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return set_err(p->c, GP_ERR_OOM, "batch plan: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  p->allocs.push_back(*ptr);
  p->bytes += (int64_t)bytes;
  return GP_OK;
}

static void plan_free_all(gp_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  p->bytes = 0;
}

#define GP_TRYB(x)              \
  do {                          \
    gp_status _s = (x);         \
    if (_s != GP_OK) return _s; \
  } while (0)
#define GP_CUDAB(p, x, where)                                   \
  do {                                                          \
    cudaError_t _e = (x);                                       \
    if (_e != cudaSuccess) return cuda_err((p)->c, _e, where);  \
  } while (0)

static BatchItems batch_view(const gp_plan* p) {
  BatchItems b;
  b.args = p->d_args;
  b.gstart = p->d_gstart;
  b.kstart = p->d_kstart;
  b.n_items = (int)p->items.size();
  b.n_gauss = p->n_gauss;
  b.n_keys = p->n_keys;
  return b;
}

// Per-item descriptors and key spaces for a tile side; uploads them.
static gp_status build_layout(gp_plan* p, int tile) {
  const int n = (int)p->items.size();
  p->tile = tile;
  p->args.assign(n, SliceArgs{});
  p->kstart.assign(n + 1, 0);
  uint64_t keys = 0;
  const float k2 = 2.0f * logf(1.0f / p->c->cfg.eps);
  size_t zoff = 0;
  for (int k = 0; k < n; ++k) {
    const gp_batch_item& it = p->items[k];
    SliceArgs& a = p->args[k];
    a.mu = it.set.mu; a.scale = it.set.scale; a.quat = it.set.quat; a.alpha = it.set.alpha;
    a.n = (int)it.set.n; a.mod = it.set.scale_mod;
    memcpy(a.Rc, p->views[k].R, sizeof(a.Rc));
    memcpy(a.tc, p->views[k].t, sizeof(a.tc));
    a.sigma2 = it.sigma_z * it.sigma_z; a.k2 = k2;
    a.S = it.S; a.H = it.H; a.W = it.W; a.tile = tile;
    a.TX = ceil_div(it.W, tile); a.TY = ceil_div(it.H, tile);
    a.zs = p->d_z + zoff;
    a.zorder = (const int*)(p->d_z + zoff + it.S);
    a.zorig = p->d_z + zoff + 2 * (size_t)it.S;
    zoff += 3 * (size_t)it.S;
    a.gbase = p->gstart[k];
    a.key_base = (uint32_t)keys;
    const int64_t img = p->img_off[k];
    a.out = it.out ? it.out : (it.target ? p->images + img : nullptr);
    a.dL_dI = it.target ? p->grads_in + img : it.dL_dI;
    const bool wants_grads = it.d_mu && (it.target || it.dL_dI);
    a.d_mu = wants_grads ? it.d_mu : nullptr;
    a.d_scale = wants_grads ? it.d_scale : nullptr;
    a.d_quat = wants_grads ? it.d_quat : nullptr;
    a.d_alpha = wants_grads ? it.d_alpha : nullptr;
    if (!wants_grads) a.dL_dI = nullptr;
    p->kstart[k] = (uint32_t)keys;
    keys += (uint64_t)it.S * a.TX * a.TY;
    if (keys >= (uint64_t)UINT32_MAX) return set_err(p->c, GP_ERR_ARG, "batch has more than 2^32 (slice, tile) keys");
  }
  p->kstart[n] = (uint32_t)keys;
  p->n_keys = (uint32_t)keys;
  GP_CUDAB(p, cudaMemcpy(p->d_args, p->args.data(), sizeof(SliceArgs) * n, cudaMemcpyHostToDevice), "upload items");
  GP_CUDAB(p, cudaMemcpy(p->d_kstart, p->kstart.data(), sizeof(uint32_t) * (n + 1), cudaMemcpyHostToDevice),
           "upload items");
  return GP_OK;
}

// Binning of the whole batch (K-pre, scan, K-emit, sort, K-range).
static gp_status enqueue_binning(gp_plan* p, cudaStream_t st) {
  const BatchItems b = batch_view(p);
  GP_CUDAB(p, cudaMemsetAsync(p->ranges, 0, (size_t)std::max<uint32_t>(p->n_keys, 1) * 8, st), "memset ranges");
  launch_slice_pre_batch(b, p->rec, p->counts, p->wsum, st);
  GP_CUDAB(p, exclusive_scan<unsigned long long>(p->wsum, p->woff, ceil_div(p->n_gauss, 32), p->total, p->scan_tmp,
                                                 st),
           "batch scan");
  if (p->cap == 0) return GP_OK;
  launch_slice_emit_batch(b, p->rec, p->woff, p->counts, p->offsets, p->cap, p->keys, p->emit_gid, st);
  int bits = 1;
  while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)p->n_keys) ++bits;
  bool in_alt = false;
  // values: Gaussian ids (read directly by the rasterisers), or the emission
  // indices by which the deterministic backward addresses its partials
  GP_CUDAB(p, radix_sort_pairs(p->keys, p->vals, p->keys_alt, p->vals_alt, p->total, p->cap, bits, p->sort_tmp, st,
                               &in_alt, p->det ? nullptr : p->emit_gid),
           "batch sort");
  p->sk = in_alt ? p->keys_alt : p->keys;
  p->sv = in_alt ? p->vals_alt : p->vals;
  launch_ranges(p->sk, p->total, p->cap, p->n_keys, p->ranges, st);
  return GP_OK;
}

static gp_status enqueue_forward(gp_plan* p, cudaStream_t st) {
  if (!p->any_fwd) return GP_OK;
  if (p->cap == 0) {  // nothing binned at plan time: the images are zero
    for (const SliceArgs& a : p->args)
      if (a.out) GP_CUDAB(p, cudaMemsetAsync(a.out, 0, (size_t)a.S * a.H * a.W * 4, st), "clear images");
    return GP_OK;
  }
  GP_CUDAB(p, cudaMemsetAsync(p->work, 0, sizeof(unsigned), st), "memset work");
  if (p->fform == GP_RASTER_PIXELS) {
    GP_CUDAB(p, launch_raster_fwd_px_batch(batch_view(p), p->tile, p->fpx, p->c->cfg.exp_mode, p->rec, p->sv,
                                           p->det ? p->emit_gid : nullptr, p->ranges, st),
             "batch forward");
    return GP_OK;
  }
  GP_CUDAB(p, launch_raster_fwd_batch(batch_view(p), p->fform == GP_RASTER_ROWS, p->tile, p->fchunk, p->ctas_f, p->c->cfg.exp_mode, p->rec, p->sv,
                                      p->det ? p->emit_gid : nullptr, p->ranges, p->work, st),
           "batch forward");
  return GP_OK;
}

static gp_status enqueue_loss(gp_plan* p, cudaStream_t st) {
  for (size_t k = 0; k < p->items.size(); ++k) {
    const gp_batch_item& it = p->items[k];
    if (!it.target) continue;
    const SliceArgs& a = p->args[k];
    launch_mse(a.out, it.target, nullptr, it.S, (int64_t)it.H * it.W, p->grads_in + p->img_off[k], it.loss,
               (float*)p->mse_tmp, st);
  }
  return GP_OK;
}

static gp_status enqueue_backward(gp_plan* p, cudaStream_t st) {
  if (!p->any_bwd) return GP_OK;
  const BatchItems b = batch_view(p);
  if (!p->det) GP_CUDAB(p, cudaMemsetAsync(p->accum, 0, (size_t)p->n_gauss * 10 * 4, st), "clear accumulators");
  if (p->cap > 0) {
    GP_CUDAB(p, cudaMemsetAsync(p->work + 1, 0, sizeof(unsigned), st), "memset work");
    if (p->bform == GP_RASTER_PIXELS)
      GP_CUDAB(p, launch_raster_bwd_px_batch(b, p->tile, p->bpx, p->c->cfg.exp_mode, p->det, p->rec, p->sv,
                                             p->det ? p->emit_gid : nullptr, p->ranges, p->accum, p->partial, st),
               "batch backward");
    else
    GP_CUDAB(p, launch_raster_bwd_batch(b, p->bform == GP_RASTER_ROWS, p->tile, p->bchunk, p->ctas_b, p->c->cfg.exp_mode, p->det, p->rec, p->sv,
                                        p->det ? p->emit_gid : nullptr, p->ranges, p->accum, p->partial, p->work + 1, st),
             "batch backward");
  }
  if (p->det) launch_det_reduce_n(p->n_gauss, p->offsets, p->counts, p->partial, p->accum, p->cap, st);
  launch_slice_bwd_pre_batch(b, p->accum, st);
  return GP_OK;
}

static gp_status enqueue_all(gp_plan* p, cudaStream_t st) {
  GP_TRYB(enqueue_binning(p, st));
  GP_TRYB(enqueue_forward(p, st));
  GP_TRYB(enqueue_loss(p, st));
  GP_TRYB(enqueue_backward(p, st));
  k_overflow_flag<<<1, 32, 0, st>>>(p->total, (unsigned long long)p->cap, p->flag);
  note_launch();
  GP_CUDAB(p, cudaMemcpyAsync(p->h_flag, p->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "flag readback");
  return cuda_err(p->c, cudaGetLastError(), "batch kernels");
}

// Pairs the batch bins with the current layout (one count, read back).
static gp_status count_pairs_now(gp_plan* p, unsigned long long* tot) {
  cudaStream_t st = p->cap_stream;
  launch_slice_pre_batch(batch_view(p), p->rec, p->counts, p->wsum, st);
  GP_CUDAB(p, exclusive_scan<unsigned long long>(p->wsum, p->woff, ceil_div(p->n_gauss, 32), p->total, p->scan_tmp,
                                                 st),
           "batch scan");
  GP_CUDAB(p, cudaMemcpyAsync(p->h_flag + 2, p->total, 8, cudaMemcpyDeviceToHost, st), "count readback");
  GP_CUDAB(p, cudaStreamSynchronize(st), "count readback");
  memcpy(tot, p->h_flag + 2, 8);
  return GP_OK;
}

static uint32_t with_headroom(unsigned long long tot) {
  const unsigned long long want = tot + tot / 4 + 65536;
  return want >= (unsigned long long)INT32_MAX ? 0u : (uint32_t)want;
}

static gp_status alloc_pairs(gp_plan* p, uint32_t cap, uint32_t n_keys) {
  const size_t P = std::max<uint32_t>(cap, 1);
  GP_TRYB(plan_alloc(p, (void**)&p->keys, P * 4));
  GP_TRYB(plan_alloc(p, (void**)&p->vals, P * 4));
  GP_TRYB(plan_alloc(p, (void**)&p->keys_alt, P * 4));
  GP_TRYB(plan_alloc(p, (void**)&p->vals_alt, P * 4));
  GP_TRYB(plan_alloc(p, (void**)&p->emit_gid, P * 4));
  GP_TRYB(plan_alloc(p, &p->sort_tmp, (size_t)radix_temp_bytes((int64_t)P)));
  GP_TRYB(plan_alloc(p, (void**)&p->ranges, (size_t)std::max<uint32_t>(n_keys, 1) * 8));
  if (p->det && p->any_bwd) GP_TRYB(plan_alloc(p, (void**)&p->partial, P * 32));
  return GP_OK;
}

static void set_ctas(gp_plan* p) {
  const int sm = p->c->sm_count;
  p->ctas_f = std::max(1, raster_batch_ctas_per_sm(p->fform == GP_RASTER_ROWS, p->tile, p->fchunk, false,
                                                   p->c->cfg.exp_mode)) * sm;
  p->ctas_b = std::max(1, raster_batch_ctas_per_sm(p->bform == GP_RASTER_ROWS, p->tile, p->bchunk, true,
                                                   p->c->cfg.exp_mode)) * sm;
}

static gp_status capture(gp_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  GP_CUDAB(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  gp_status s = enqueue_all(p, p->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
  if (s != GP_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_err(p->c, e, "end capture");
  p->graph = g;
  GP_CUDAB(p, cudaGraphInstantiate(&p->exec, g, 0), "graph instantiate");
  return GP_OK;
}

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// Times one phase: a warm-up, then `reps` repetitions.
template <class F>
static double time_phase(gp_plan* p, F&& f, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  f();
  cudaEventRecord(a, p->cap_stream);
  for (int r = 0; r < reps; ++r) f();
  cudaEventRecord(b, p->cap_stream);
  const double ms = elapsed(a, b) / reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGetLastError();
  return ms;
}

// One rasteriser configuration of a pass: form, staging chunk (block-culled)
// or pixels per thread (per-thread).
struct PassCfg {
  int form, chunk, px;
};

static std::vector<PassCfg> pass_candidates(const gp_plan* p, bool backward) {
  std::vector<PassCfg> c;
  for (int ch : backward ? std::vector<int>{32, 64, 128} : std::vector<int>{64, 128, 256})
    c.push_back({GP_RASTER_BLOCK, ch, 0});
  if (p->c->cfg.exp_mode == GP_EXP_POLY_ROW) return c;  // block-culled only
  c.push_back({GP_RASTER_ROWS, backward ? p->bchunk : p->fchunk, 0});
  std::vector<int> pxs;
  if (p->tile == 16) pxs = backward ? std::vector<int>{2, 4, 8} : std::vector<int>{1, 2, 4};
  else pxs = backward ? std::vector<int>{2} : std::vector<int>{1, 2};
  for (int px : pxs) c.push_back({GP_RASTER_PIXELS, backward ? p->bchunk : p->fchunk, px});
  return c;
}

static gp_status autotune(gp_plan* p, const std::vector<int>& tiles, const std::vector<uint32_t>& caps) {
  double best = 1e30;
  int bt = p->tile;
  PassCfg bf{p->fform, p->fchunk, p->fpx}, bb{p->bform, p->bchunk, p->bpx};
  for (size_t t = 0; t < tiles.size(); ++t) {
    GP_TRYB(build_layout(p, tiles[t]));
    p->cap = caps[t];
    if (p->cap == 0) continue;
    GP_TRYB(enqueue_binning(p, p->cap_stream));  // also leaves the binning for the timings below
    const double t_bin = time_phase(p, [&] { enqueue_binning(p, p->cap_stream); }, 2);
    double t_f = 0.0, t_b = 0.0;
    PassCfg cf{p->fform, p->fchunk, p->fpx}, cb{p->bform, p->bchunk, p->bpx};
    if (p->any_fwd) {
      t_f = 1e30;
      for (const PassCfg& k : pass_candidates(p, false)) {
        p->fform = k.form;
        p->fchunk = k.chunk;
        p->fpx = k.px;
        set_ctas(p);
        const double ms = time_phase(p, [&] { enqueue_forward(p, p->cap_stream); }, 2);
        if (ms < t_f) { t_f = ms; cf = k; }
      }
    }
    if (p->any_bwd) {
      enqueue_loss(p, p->cap_stream);
      t_b = 1e30;
      for (const PassCfg& k : pass_candidates(p, true)) {
        p->bform = k.form;
        p->bchunk = k.chunk;
        p->bpx = k.px;
        set_ctas(p);
        const double ms = time_phase(p, [&] { enqueue_backward(p, p->cap_stream); }, 2);
        if (ms < t_b) { t_b = ms; cb = k; }
      }
    }
    const double tot = t_bin + t_f + t_b;
    if (tot < best) { best = tot; bt = tiles[t]; bf = cf; bb = cb; }
  }
  GP_CUDAB(p, cudaStreamSynchronize(p->cap_stream), "autotune");
  p->fform = bf.form;
  p->fchunk = bf.chunk;
  p->fpx = bf.px;
  p->bform = bb.form;
  p->bchunk = bb.chunk;
  p->bpx = bb.px;
  for (size_t t = 0; t < tiles.size(); ++t)
    if (tiles[t] == bt) p->cap = caps[t];
  return build_layout(p, bt);
}

static gp_status plan_build(gp_plan* p) {
  Ctx* c = p->c;
  const int n = (int)p->items.size();
  // validate items and lay out Gaussians, planes and plan-owned images
  p->gstart.assign(n + 1, 0);
  p->img_off.assign(n, 0);
  p->views.assign(n, View{});
  int64_t gs = 0, imgs = 0, zs = 0, mse_tmp = 1;
  for (int k = 0; k < n; ++k) {
    const gp_batch_item& it = p->items[k];
    if (it.set.n < 0 || (it.set.n > 0 && (!it.set.mu || !it.set.scale || !it.set.quat || !it.set.alpha)))
      return set_err(c, GP_ERR_ARG, "batch item " + std::to_string(k) + ": bad Gaussian set");
    if (it.set.n > 0 && ((uintptr_t)it.set.quat & 15u)) return set_err(c, GP_ERR_ARG, "quat must be 16-byte aligned");
    if (!(it.set.scale_mod > 0.0f)) return set_err(c, GP_ERR_ARG, "scale_mod must be > 0");
    if (it.S < 0 || it.H <= 0 || it.W <= 0 || (it.S > 0 && !it.z))
      return set_err(c, GP_ERR_ARG, "batch item " + std::to_string(k) + ": bad slice stack");
    if (!(it.sigma_z > 0.0f) || !isfinite(it.sigma_z))
      return set_err(c, GP_ERR_ARG, "batch item " + std::to_string(k) + ": bad sigma_z");
    if (it.view ? !check_view(it.view, &p->views[k]) : !axis_view(it.axis, &p->views[k]))
      return set_err(c, GP_ERR_ARG, "batch item " + std::to_string(k) + ": bad axis or view");
    if ((int64_t)it.S * it.H * it.W > (int64_t)INT32_MAX) return set_err(c, GP_ERR_ARG, "item image too large");
    for (int s = 0; s < it.S; ++s)
      if (!isfinite(it.z[s])) return set_err(c, GP_ERR_ARG, "z contains a non-finite value");
    if (it.d_mu && (!it.d_scale || !it.d_quat || !it.d_alpha || ((uintptr_t)it.d_quat & 15u)))
      return set_err(c, GP_ERR_ARG, "batch item " + std::to_string(k) + ": bad gradient pointers");
    p->gstart[k] = (int)gs;
    gs += it.set.n;
    if (gs > (int64_t)INT32_MAX - 1) return set_err(c, GP_ERR_ARG, "batch has too many Gaussians");
    p->img_off[k] = imgs;
    if (it.target) {
      imgs += (int64_t)it.S * it.H * it.W;
      mse_tmp = std::max<int64_t>(mse_tmp, mse_tmp_floats(it.S, (int64_t)it.H * it.W));
    }
    zs += 3 * (int64_t)it.S;
    p->any_fwd = p->any_fwd || it.out || it.target;
    p->any_bwd = p->any_bwd || (it.d_mu && (it.target || it.dL_dI));
  }
  p->gstart[n] = (int)gs;
  p->n_gauss = (int)gs;
  p->det = c->cfg.deterministic != 0;
  // forms without autotuning: as the plain calls choose them on slice planes
  const bool rows_ok = c->cfg.exp_mode != GP_EXP_POLY_ROW;
  p->fform = (c->cfg.raster != GP_RASTER_BLOCK && rows_ok) ? GP_RASTER_ROWS : GP_RASTER_BLOCK;
  p->bform = (c->cfg.raster == GP_RASTER_ROWS && rows_ok) ? GP_RASTER_ROWS : GP_RASTER_BLOCK;
  // a context with a per-thread rasteriser keeps it
  if (c->cfg.fwd_px > 0) { p->fform = GP_RASTER_PIXELS; p->fpx = c->cfg.fwd_px; }
  if (c->cfg.bwd_px > 0) { p->bform = GP_RASTER_PIXELS; p->bpx = c->cfg.bwd_px; }
  // fixed allocations
  GP_TRYB(plan_alloc(p, (void**)&p->d_args, sizeof(SliceArgs) * n));
  GP_TRYB(plan_alloc(p, (void**)&p->d_gstart, sizeof(int) * (n + 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->d_kstart, sizeof(uint32_t) * (n + 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->d_z, sizeof(float) * std::max<int64_t>(zs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->rec, sizeof(SliceRec) * std::max<int64_t>(gs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->counts, 8 * std::max<int64_t>(gs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->offsets, 8 * std::max<int64_t>(gs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->wsum, 8 * std::max<int64_t>((gs + 31) / 32, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->woff, 8 * std::max<int64_t>((gs + 31) / 32, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->total, 64));
  GP_TRYB(plan_alloc(p, &p->scan_tmp, (size_t)scan_temp_bytes(std::max<int64_t>(gs, 1))));
  GP_TRYB(plan_alloc(p, (void**)&p->accum, 40 * std::max<int64_t>(gs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->images, 4 * std::max<int64_t>(imgs, 1)));
  GP_TRYB(plan_alloc(p, (void**)&p->grads_in, 4 * std::max<int64_t>(imgs, 1)));
  GP_TRYB(plan_alloc(p, &p->mse_tmp, 4 * (size_t)mse_tmp));
  GP_TRYB(plan_alloc(p, (void**)&p->work, 64));
  GP_TRYB(plan_alloc(p, (void**)&p->flag, 64));
  GP_CUDAB(p, cudaMemcpy(p->d_gstart, p->gstart.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice), "upload");
  // planes per item: sorted positions, their slice indices (as int bits), positions by index
  std::vector<float> zbuf((size_t)std::max<int64_t>(zs, 1));
  size_t zo = 0;
  for (int k = 0; k < n; ++k) {
    const gp_batch_item& it = p->items[k];
    std::vector<int> order(it.S);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return it.z[i] < it.z[j]; });
    for (int j = 0; j < it.S; ++j) {
      zbuf[zo + j] = it.z[order[j]];
      memcpy(&zbuf[zo + it.S + j], &order[j], 4);
      zbuf[zo + 2 * it.S + j] = it.z[j];
    }
    zo += 3 * (size_t)it.S;
  }
  GP_CUDAB(p, cudaMemcpy(p->d_z, zbuf.data(), 4 * zbuf.size(), cudaMemcpyHostToDevice), "upload planes");
  // candidate tile sides: count pairs for each, then size the pair buffers for the largest
  std::vector<int> tiles;
  if (p->flags & GP_BATCH_AUTOTUNE) tiles = {16, 8};
  else tiles = {c->cfg.tile == 8 ? 8 : 16};
  std::vector<uint32_t> caps;
  uint32_t maxcap = 0, maxkeys = 0;
  for (int t : tiles) {
    GP_TRYB(build_layout(p, t));
    unsigned long long tot = 0;
    GP_TRYB(count_pairs_now(p, &tot));
    const uint32_t cap = tot == 0 ? 0u : with_headroom(tot);
    if (tot > 0 && cap == 0) return set_err(c, GP_ERR_OVERFLOW, "batch has more than 2^31 binned pairs; split it");
    caps.push_back(cap);
    maxcap = std::max(maxcap, cap);
    maxkeys = std::max(maxkeys, p->n_keys);
  }
  GP_TRYB(alloc_pairs(p, maxcap, maxkeys));
  if (tiles.size() > 1) {
    GP_TRYB(autotune(p, tiles, caps));
  } else {
    p->cap = caps[0];
  }
  set_ctas(p);
  return capture(p);
}

}  // namespace gp

extern "C" {

gp_status gp_batch_plan(gp_ctx* ctx, const gp_batch_item* items, int n, int flags, gp_plan** out) {
  if (!ctx || !out) return GP_ERR_ARG;
  *out = nullptr;
  Ctx* c = &ctx->impl;
  if (n <= 0 || !items) return set_err(c, GP_ERR_ARG, "batch needs at least one item");
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
  gp_plan* p = new (std::nothrow) gp_plan();
  if (!p) return GP_ERR_OOM;
  p->c = c;
  p->items.assign(items, items + n);
  p->flags = flags;
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_flag, 64);
  if (e != cudaSuccess) {
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
    return cuda_err(c, e, "batch plan");
  }
  *p->h_flag = 0;
  gp_status s = plan_build(p);
  if (s != GP_OK) {
    cudaStreamSynchronize(p->cap_stream);
    plan_free_all(p);
    cudaStreamDestroy(p->cap_stream);
    cudaFreeHost(p->h_flag);
    delete p;
    return s;
  }
  *out = p;
  return GP_OK;
}

gp_status gp_batch_run(gp_plan* p, void* stream) {
  if (!p || !p->exec) return GP_ERR_ARG;
  gp::NvtxRange range("gp:batch_run");
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_err(p->c, e, "graph launch");
  return GP_OK;
}

gp_status gp_batch_wait(gp_plan* p, void* stream) {
  if (!p) return GP_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_err(p->c, e, "batch wait");
  if (*p->h_flag) return set_err(p->c, GP_ERR_OVERFLOW, "batch pairs exceeded the planned buffers; re-plan");
  return check_after(p->c, (cudaStream_t)stream);
}

gp_status gp_batch_info(gp_plan* p, gp_batch_config* out) {
  if (!p || !out) return GP_ERR_ARG;
  out->pair_capacity = p->cap;
  out->device_bytes = p->bytes;
  out->tile = p->tile;
  out->fwd_raster = p->fform;
  out->bwd_raster = p->bform;
  out->fwd_chunk = p->fform == GP_RASTER_BLOCK ? p->fchunk : 0;
  out->bwd_chunk = p->bform == GP_RASTER_BLOCK ? p->bchunk : 0;
  out->fwd_px = p->fform == GP_RASTER_PIXELS ? p->fpx : 0;
  out->bwd_px = p->bform == GP_RASTER_PIXELS ? p->bpx : 0;
  return GP_OK;
}

gp_status gp_batch_destroy(gp_plan* p) {
  if (!p) return GP_ERR_ARG;
  cudaStreamSynchronize(p->cap_stream);
  cudaDeviceSynchronize();
  plan_free_all(p);
  cudaStreamDestroy(p->cap_stream);
  cudaFreeHost(p->h_flag);
  delete p;
  return GP_OK;
}

}  // extern "C"
