// runtime.cu -- C ABI of the slice projection library: context, workspace pool,
// argument checking and the host sequencing of the render / backward /
// voxelize pipelines.  Every arithmetic step runs in the kernels of slice.cu,
// raster.cu and sort.cu (the voxelizer is the slice path over the grid's
// z-planes with sigma_z = 0 and amplitude alpha).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gp_internal.h"
#include "slice.cuh"

namespace gp {

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

static const char* phase_range_name(int phase) {
  static const char* const names[] = {"gp:bin", "gp:fwd", "gp:bwd", "gp:bwd_pre",
                                      "gp:loss", "gp:vox_fwd", "gp:vox_bwd", "gp:opt"};
  return phase >= 0 && phase < (int)(sizeof(names) / sizeof(names[0])) ? names[phase] : "gp:phase";
}

static std::atomic<int64_t> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

static cudaEvent_t pooled_event(Ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseTimer::PhaseTimer(Ctx* c, int phase, cudaStream_t st)
    : range_(phase_range_name(phase)), c_(c), phase_(phase), st_(st) {
  if (!((c->timing >> phase) & 1u)) return;
  start_ = pooled_event(c);
  if (start_ && cudaEventRecord(start_, st) != cudaSuccess) {
    cudaGetLastError();
    c->event_pool.push_back(start_);
    start_ = nullptr;
  }
  l0_ = launch_count();
}

PhaseTimer::~PhaseTimer() {
  if (!start_) return;
  cudaEvent_t stop = pooled_event(c_);
  if (!stop || cudaEventRecord(stop, st_) != cudaSuccess) {
    cudaGetLastError();
    c_->event_pool.push_back(start_);
    if (stop) c_->event_pool.push_back(stop);
    return;
  }
  c_->events.push_back(PhaseEvent{phase_, start_, stop, launch_count() - l0_});
}

gp_status set_err(Ctx* c, gp_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

gp_status cuda_err(Ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return GP_OK;
  cudaGetLastError();  // clear the (non-sticky) error so the context stays usable
  if (e == cudaErrorMemoryAllocation) return set_err(c, GP_ERR_OOM, std::string(where) + ": out of device memory");
  return set_err(c, GP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Frees every workspace buffer of the context (and forgets the binning they
// held).  cudaFree waits for the work already queued on the device, so this is
// safe while kernels of the failing call are still in flight.
void ws_release_all(Ctx* c) {
  BinBufs& b = c->b;
  DevBuf* all[] = {&b.rec, &b.counts, &b.offsets, &b.total, &b.keys, &b.vals, &b.keys_alt, &b.vals_alt,
                   &b.emit_gid, &b.ranges, &b.scan_tmp, &b.sort_tmp, &b.zs, &b.zorder, &b.zorig,
                   &b.accum, &b.partial, &b.loss_tmp, &b.codec};
  for (DevBuf* d : all) ws_release(c, *d);
  c->bin_key.valid = false;
}

// Grows buf to at least `bytes` (by 25 % steps).  A request past the
// context's workspace limit, or a failed cudaMalloc, frees the whole workspace
// before it returns GP_ERR_OOM (every caller then returns the error at once),
// so the context is left empty and later calls that fit still run.
gp_status ws_reserve(Ctx* c, DevBuf& buf, size_t bytes) {
  if (bytes <= buf.bytes) return GP_OK;
  size_t want = std::max(bytes, (size_t)(buf.bytes * 1.25));
  want = (want + 255) & ~(size_t)255;
  int64_t limit = c->cfg.workspace_limit;
  if (limit > 0 && c->ws_bytes - (int64_t)buf.bytes + (int64_t)want > limit) {
    want = (bytes + 255) & ~(size_t)255;
    if (c->ws_bytes - (int64_t)buf.bytes + (int64_t)want > limit) {
      ws_release_all(c);
      return set_err(c, GP_ERR_OOM, "workspace limit exceeded (" + std::to_string(limit) + " bytes)");
    }
  }
  if (buf.ptr) {
    cudaError_t e = cudaFree(buf.ptr);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaFree");
    c->ws_bytes -= (int64_t)buf.bytes;
    buf.ptr = nullptr;
    buf.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&buf.ptr, want);
  if (e != cudaSuccess) {
    buf.ptr = nullptr;
    cudaGetLastError();
    ws_release_all(c);
    return set_err(c, GP_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
  }
  buf.bytes = want;
  c->ws_bytes += (int64_t)want;
  return GP_OK;
}

void ws_release(Ctx* c, DevBuf& buf) {
  if (buf.ptr) {
    cudaFree(buf.ptr);
    c->ws_bytes -= (int64_t)buf.bytes;
  }
  buf.ptr = nullptr;
  buf.bytes = 0;
}

#define GP_TRY(x)               \
  do {                          \
    gp_status _s = (x);         \
    if (_s != GP_OK) return _s; \
  } while (0)
#define GP_CUDA(c, x, where)                               \
  do {                                                     \
    cudaError_t _e = (x);                                  \
    if (_e != cudaSuccess) return cuda_err(c, _e, where);  \
  } while (0)

gp_status check_after(Ctx* c, cudaStream_t st) {
#ifdef GP_CHECK
  GP_CUDA(c, cudaStreamSynchronize(st), "bounds check");
  const char* files[] = {"raster.cu", "slice.cu", "sort.cu"};
  const unsigned long long words[] = {check_read_raster(), check_read_slice(), check_read_sort()};
  for (int k = 0; k < 3; ++k)
    if (words[k])
      return set_err(c, GP_ERR_STATE, std::string("bounds check failed in ") + files[k] + " at site " +
                                           std::to_string(words[k] >> 40) + ", index " +
                                           std::to_string((long long)(words[k] & ((1ull << 40) - 1ull))));
#else
  (void)c;
  (void)st;
#endif
  return GP_OK;
}

constexpr int kPutWords = 720;
struct PutArgs {
  uint32_t* dst[3];
  int n[3];
  uint32_t w[kPutWords];
};

__global__ void k_put_words(PutArgs p) {
  int o = 0;
  for (int s = 0; s < 3; ++s) {
    for (int i = threadIdx.x; i < p.n[s]; i += blockDim.x) p.dst[s][i] = p.w[o + i];
    o += p.n[s];
  }
}

cudaError_t put_words(cudaStream_t st, int k, uint32_t* const* dst, const void* const* src, const int* n) {
  int tot = 0;
  for (int s = 0; s < k; ++s) tot += n[s];
  if (k <= 3 && tot <= kPutWords) {
    if (tot == 0) return cudaSuccess;
    PutArgs p{};
    int o = 0;
    for (int s = 0; s < k; ++s) {
      p.dst[s] = dst[s];
      p.n[s] = n[s];
      memcpy(p.w + o, src[s], (size_t)n[s] * 4);
      o += n[s];
    }
    k_put_words<<<1, 256, 0, st>>>(p);
    note_launch();
    return cudaGetLastError();
  }
  for (int s = 0; s < k; ++s) {
    if (n[s] == 0) continue;
    cudaError_t e = cudaMemcpyAsync(dst[s], src[s], (size_t)n[s] * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static gp_status check_set(Ctx* c, const gp_set* s) {
  if (!s) return set_err(c, GP_ERR_ARG, "set is NULL");
  if (s->n < 0 || s->n > (int64_t)INT32_MAX - 1) return set_err(c, GP_ERR_ARG, "set size out of range");
  if (s->n > 0 && (!s->mu || !s->scale || !s->quat || !s->alpha))
    return set_err(c, GP_ERR_ARG, "set has a NULL parameter pointer");
  if (s->n > 0 && !aligned16(s->quat)) return set_err(c, GP_ERR_ARG, "quat must be 16-byte aligned");
  if (!(s->scale_mod > 0.0f) || !isfinite(s->scale_mod)) return set_err(c, GP_ERR_ARG, "scale_mod must be > 0");
  return GP_OK;
}

static int tile_of(const Ctx* c) { return c->cfg.tile == 8 ? 8 : 16; }
static int fwd_px(const Ctx* c) { return c->cfg.fwd_px; }
static int bwd_px(const Ctx* c) { return c->cfg.bwd_px; }

// Sorts the emitted (key, value) pairs and finds the tile ranges.  The values
// are the Gaussian ids when first_vals is the emission-to-Gaussian map (the
// rasterisers then read them directly), or the emission indices when it is
// NULL (the deterministic backward indexes its per-pair partials by them).
static gp_status sort_and_range(Ctx* c, uint32_t P, int64_t nkeys, cudaStream_t st, const uint32_t** sorted_vals,
                                const uint32_t* first_vals) {
  BinBufs& b = c->b;
  int bits = 1;
  while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)nkeys) ++bits;
  bool in_alt = false;
  GP_CUDA(c, radix_sort_pairs((uint32_t*)b.keys.ptr, (uint32_t*)b.vals.ptr, (uint32_t*)b.keys_alt.ptr,
                              (uint32_t*)b.vals_alt.ptr, (const unsigned long long*)b.total.ptr, P, bits,
                              b.sort_tmp.ptr, st, &in_alt, first_vals),
          "radix sort");
  const uint32_t* sk = (const uint32_t*)(in_alt ? b.keys_alt.ptr : b.keys.ptr);
  *sorted_vals = (const uint32_t*)(in_alt ? b.vals_alt.ptr : b.vals.ptr);
  launch_ranges(sk, (const unsigned long long*)b.total.ptr, P, (uint32_t)nkeys, (uint2*)b.ranges.ptr, st);
  return GP_OK;
}

static gp_status reserve_pairs(Ctx* c, uint32_t P) {
  BinBufs& b = c->b;
  GP_TRY(ws_reserve(c, b.keys, (size_t)P * 4));
  GP_TRY(ws_reserve(c, b.vals, (size_t)P * 4));
  GP_TRY(ws_reserve(c, b.keys_alt, (size_t)P * 4));
  GP_TRY(ws_reserve(c, b.vals_alt, (size_t)P * 4));
  GP_TRY(ws_reserve(c, b.emit_gid, (size_t)P * 4));
  GP_TRY(ws_reserve(c, b.sort_tmp, (size_t)radix_temp_bytes(P)));
  return GP_OK;
}

// Scan of the per-warp pair totals (K-emit derives each Gaussian's offset).
static cudaError_t scan_warp_totals(Ctx* c, int n, cudaStream_t st) {
  BinBufs& b = c->b;
  return exclusive_scan<unsigned long long>((unsigned long long*)b.wsum.ptr, (unsigned long long*)b.woff.ptr,
                                            ceil_div(n, 32), (unsigned long long*)b.total.ptr, b.scan_tmp.ptr, st);
}

// The scan and the one host readback of the total.
static gp_status scan_counts(Ctx* c, int n, cudaStream_t st, uint32_t* P) {
  BinBufs& b = c->b;
  GP_CUDA(c, scan_warp_totals(c, n, st), "pair scan");
  GP_CUDA(c, cudaMemcpyAsync(c->h_total, b.total.ptr, 8, cudaMemcpyDeviceToHost, st), "pair count readback");
  GP_CUDA(c, cudaStreamSynchronize(st), "pair count readback");
  unsigned long long tot = *c->h_total;
  if (tot >= (unsigned long long)INT32_MAX)
    return set_err(c, GP_ERR_OVERFLOW, "more than 2^31 binned pairs in one call; split the call");
  *P = (uint32_t)tot;
  return GP_OK;
}

// Pairs the context's pair buffers (and the sort's scratch) hold, 0 if none.
static uint32_t pair_capacity(Ctx* c) {
  const BinBufs& b = c->b;
  size_t bytes = std::min({b.keys.bytes, b.vals.bytes, b.keys_alt.bytes, b.vals_alt.bytes, b.emit_gid.bytes});
  uint32_t cap = (uint32_t)std::min<size_t>(bytes / 4, (size_t)INT32_MAX - 1);
  while (cap > 0 && (size_t)radix_temp_bytes(cap) > b.sort_tmp.bytes) cap -= std::max<uint32_t>(cap / 64, 1);
  return cap;
}

// Completes a speculative binning (see bin_slices): waits for the pair count's
// copy and sets the binned pair count, or sets *redo when the pairs did not
// fit the buffers the emission and sort were sized by (the caller then bins
// again without speculation and repeats its rasteriser).
static gp_status finish_bin(Ctx* c, bool* redo) {
  *redo = false;
  if (!c->bin_pending) return GP_OK;
  c->bin_pending = false;
  GP_CUDA(c, cudaEventSynchronize(c->bin_ev), "pair count readback");
  const unsigned long long tot = *c->h_total;
  if (tot >= (unsigned long long)INT32_MAX) {
    c->bin_key.valid = false;
    return set_err(c, GP_ERR_OVERFLOW, "more than 2^31 binned pairs in one call; split the call");
  }
  if (tot > c->bin_cap) {
    c->bin_key.valid = false;
    *redo = true;
    return GP_OK;
  }
  c->bin_pairs = (uint32_t)tot;
  c->last_pairs = (int64_t)tot;
  c->last_issued = (int64_t)tot * c->bin_key.tile * c->bin_key.tile;
  return GP_OK;
}

// Bins the set's (Gaussian, slice, tile) pairs of a slice stack: K-pre, scan,
// one count readback, K-emit, radix sort, K-range.  On return the context's
// buffers hold the records, the sorted emission indices and the tile ranges,
// and *a describes the launch.
// vox: the planes of the voxelizer (Eq. 12): sigma_z = 0 and amplitude alpha.
// speculate: when the context already holds pair buffers, emit and sort into
// their capacity without waiting for the pair count (the sort and the tile
// ranges take the count from device memory); the count's copy is then pending,
// *pairs_out is the capacity, and the caller queues its rasteriser and calls
// finish_bin, so the host's wait for the count overlaps the device's work
// instead of stalling the device between the scan and the emission.
static gp_status bin_slices(Ctx* c, const gp_set* set, const float* z, int S, int H, int W, float sigma_z,
                            const View& view, cudaStream_t st, SliceArgs* a, uint32_t* pairs_out,
                            const uint32_t** sorted_vals, bool vox = false, bool speculate = false) {
  if (c->bin_pending) {  // an earlier speculative binning whose caller failed before finishing it
    c->bin_pending = false;
    GP_CUDA(c, cudaEventSynchronize(c->bin_ev), "pair count readback");
  }
  if (S < 0 || H <= 0 || W <= 0) return set_err(c, GP_ERR_ARG, "need S >= 0, H > 0, W > 0");
  if (S > 0 && !z) return set_err(c, GP_ERR_ARG, "z is NULL");
  if (vox) sigma_z = 0.0f;
  else if (!(sigma_z > 0.0f) || !isfinite(sigma_z)) return set_err(c, GP_ERR_ARG, "sigma_z must be in (0, inf)");
  if ((int64_t)S * H * W > (int64_t)INT32_MAX) return set_err(c, GP_ERR_ARG, "S*H*W exceeds 2^31");
  for (int s = 0; s < S; ++s)
    if (!isfinite(z[s])) return set_err(c, GP_ERR_ARG, "z contains a non-finite value");
  PhaseTimer timer(c, GP_PHASE_BIN, st);
  c->bin_key.valid = false;  // until this binning completes
  const int tile = tile_of(c);
  const int TX = ceil_div(W, tile), TY = ceil_div(H, tile);
  const int64_t nkeys = (int64_t)S * TX * TY;
  if (nkeys >= (int64_t)UINT32_MAX) return set_err(c, GP_ERR_ARG, "too many (slice, tile) bins");
  BinBufs& b = c->b;
  const int n = (int)set->n;
  // slice positions: sorted copy + order (host), uploaded once per call
  std::vector<int> order(S);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return z[i] < z[j]; });
  std::vector<float> zs(S);
  for (int j = 0; j < S; ++j) zs[j] = z[order[j]];
  GP_TRY(ws_reserve(c, b.zs, (size_t)std::max(S, 1) * 4));
  GP_TRY(ws_reserve(c, b.zorder, (size_t)std::max(S, 1) * 4));
  GP_TRY(ws_reserve(c, b.zorig, (size_t)std::max(S, 1) * 4));
  if (S > 0) {
    uint32_t* dst[3] = {(uint32_t*)b.zs.ptr, (uint32_t*)b.zorder.ptr, (uint32_t*)b.zorig.ptr};
    const void* src[3] = {zs.data(), order.data(), z};
    const int cnt[3] = {S, S, S};
    GP_CUDA(c, put_words(st, 3, dst, src, cnt), "upload z");
  }
  SliceArgs& A = *a;
  A = SliceArgs{};
  A.mu = set->mu; A.scale = set->scale; A.quat = set->quat; A.alpha = set->alpha;
  A.n = n; A.mod = set->scale_mod; A.sigma2 = sigma_z * sigma_z;
  A.vox = vox ? 1 : 0;
  memcpy(A.Rc, view.R, sizeof(A.Rc));
  memcpy(A.tc, view.t, sizeof(A.tc));
  A.k2 = 2.0f * logf(1.0f / c->cfg.eps);
  A.zs = (const float*)b.zs.ptr; A.zorder = (const int*)b.zorder.ptr; A.zorig = (const float*)b.zorig.ptr;
  A.S = S; A.H = H; A.W = W; A.tile = tile; A.TX = TX; A.TY = TY;
  GP_TRY(ws_reserve(c, b.rec, (size_t)std::max(n, 1) * sizeof(SliceRec)));
  GP_TRY(ws_reserve(c, b.counts, (size_t)std::max(n, 1) * 8));
  GP_TRY(ws_reserve(c, b.offsets, (size_t)std::max(n, 1) * 8));
  GP_TRY(ws_reserve(c, b.wsum, (size_t)std::max(ceil_div(n, 32), 1) * 8));
  GP_TRY(ws_reserve(c, b.woff, (size_t)std::max(ceil_div(n, 32), 1) * 8));
  GP_TRY(ws_reserve(c, b.total, 64));
  GP_TRY(ws_reserve(c, b.scan_tmp, (size_t)scan_temp_bytes(std::max(n, 1))));
  GP_TRY(ws_reserve(c, b.ranges, (size_t)std::max<int64_t>(nkeys, 1) * 8));
  GP_CUDA(c, cudaMemsetAsync(b.ranges.ptr, 0, (size_t)std::max<int64_t>(nkeys, 1) * 8, st), "memset ranges");
  uint32_t P = 0;
  bool spec = false;
  if (n > 0 && S > 0) {
    launch_slice_pre(A, (SliceRec*)b.rec.ptr, (unsigned long long*)b.counts.ptr, (unsigned long long*)b.wsum.ptr, st);
    // the speculative capacity: the buffers' capacity, but at most a quarter
    // more than the last binning's count (the sort's grids and scans are sized
    // by it)
    uint32_t cap = speculate ? pair_capacity(c) : 0u;
    if (cap > 0 && c->last_pairs > 0)
      cap = (uint32_t)std::min<int64_t>(cap, std::max<int64_t>(c->last_pairs + c->last_pairs / 4, 4096));
    if (cap > 0) {
      GP_CUDA(c, scan_warp_totals(c, n, st), "pair scan");
      // the count's copy runs on the context's side stream as soon as the scan
      // is done, beside the emission and the sort
      GP_CUDA(c, cudaEventRecord(c->scan_ev, st), "pair count readback");
      GP_CUDA(c, cudaStreamWaitEvent(c->side_st, c->scan_ev, 0), "pair count readback");
      GP_CUDA(c, cudaMemcpyAsync(c->h_total, b.total.ptr, 8, cudaMemcpyDeviceToHost, c->side_st),
              "pair count readback");
      GP_CUDA(c, cudaEventRecord(c->bin_ev, c->side_st), "pair count readback");
      c->bin_pending = true;
      P = cap;
      spec = true;
    } else {
      GP_TRY(scan_counts(c, n, st, &P));
    }
  } else if (n > 0) {
    GP_CUDA(c, cudaMemsetAsync(b.counts.ptr, 0, (size_t)n * 8, st), "clear counts");
    GP_CUDA(c, cudaMemsetAsync(b.offsets.ptr, 0, (size_t)n * 8, st), "clear offsets");
  }
  *sorted_vals = nullptr;
  if (P > 0) {
    // an eighth more than this call needs, so that the next calls' counts
    // usually fit the buffers a speculative binning is sized by
    if (!spec) GP_TRY(reserve_pairs(c, (uint32_t)std::min<uint64_t>((uint64_t)P + P / 8, (uint64_t)INT32_MAX - 1)));
    launch_slice_emit(A, (const SliceRec*)b.rec.ptr, (const unsigned long long*)b.woff.ptr,
                      (const unsigned long long*)b.counts.ptr, (unsigned long long*)b.offsets.ptr,
                      (uint32_t*)b.keys.ptr, (uint32_t*)b.emit_gid.ptr, st, P);
    c->bin_gid_vals = c->cfg.deterministic == 0;
    GP_TRY(sort_and_range(c, P, nkeys, st, sorted_vals,
                          c->bin_gid_vals ? (const uint32_t*)b.emit_gid.ptr : nullptr));
  }
  if (spec) c->bin_cap = P;
  *pairs_out = P;
  c->last_pairs = P;
  c->last_issued = (int64_t)P * tile * tile;
  BinKey& k = c->bin_key;
  k.valid = true;
  k.mu = set->mu; k.scale = set->scale; k.quat = set->quat; k.alpha = set->alpha;
  k.n = set->n; k.mod = set->scale_mod; k.sigma_z = sigma_z;
  k.z.assign(z, z + S);
  k.S = S; k.H = H; k.W = W; k.view = view; k.tile = tile;
  c->bin_pairs = P;
  c->bin_vals = *sorted_vals;
  static_assert(sizeof(SliceArgs) <= sizeof(c->bin_args), "SliceArgs too large");
  memcpy(c->bin_args, a, sizeof(SliceArgs));
  return cuda_err(c, cudaGetLastError(), "binning kernels");
}

// True if the context still holds a binning made with exactly these arguments.
static bool bins_match(const Ctx* c, const gp_set* set, const float* z, int S, int H, int W, float sigma_z,
                       const View& view) {
  const BinKey& k = c->bin_key;
  if (!k.valid || k.mu != set->mu || k.scale != set->scale || k.quat != set->quat || k.alpha != set->alpha ||
      k.n != set->n || k.mod != set->scale_mod || k.sigma_z != sigma_z || k.S != S || k.H != H || k.W != W ||
      !same_view(k.view, view) || k.tile != tile_of(c))
    return false;
  for (int s = 0; s < S; ++s)
    if (k.z[s] != z[s]) return false;
  return true;
}

static gp_status check_grads(Ctx* c, int64_t n, float* d_mu, float* d_scale, float* d_quat, float* d_alpha) {
  if (n > 0 && (!d_mu || !d_scale || !d_quat || !d_alpha)) return set_err(c, GP_ERR_ARG, "gradient pointer is NULL");
  if (n > 0 && !aligned16(d_quat)) return set_err(c, GP_ERR_ARG, "d_quat must be 16-byte aligned");
  return GP_OK;
}

bool axis_view(int axis, View* v) {
  if (axis < 0 || axis > 2) return false;
  memset(v, 0, sizeof(*v));
  for (int j = 0; j < 3; ++j) v->R[3 * j + axis_perm(axis, j)] = 1.0f;
  return true;
}

bool check_view(const gp_view* in, View* out) {
  if (!in) return false;
  for (int k = 0; k < 9; ++k)
    if (!isfinite(in->R[k])) return false;
  for (int k = 0; k < 3; ++k)
    if (!isfinite(in->t[k])) return false;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      double d = 0.0;
      for (int k = 0; k < 3; ++k) d += (double)in->R[3 * r + k] * (double)in->R[3 * q + k];
      if (fabs(d - (r == q ? 1.0 : 0.0)) > 1e-3) return false;
    }
  memcpy(out->R, in->R, sizeof(out->R));
  memcpy(out->t, in->t, sizeof(out->t));
  return true;
}

bool same_view(const View& a, const View& b) { return memcmp(&a, &b, sizeof(View)) == 0; }

}  // namespace gp

using namespace gp;

extern "C" {

gp_status gp_config_default(gp_config* cfg) {
  if (!cfg) return GP_ERR_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->eps = 1e-6f;
  cfg->deterministic = 0;
  cfg->exp_mode = GP_EXP_POLY;
  cfg->tile = 16;
  cfg->fwd_px = 0;
  cfg->bwd_px = 0;
  cfg->workspace_limit = 0;
  cfg->reuse_bins = 0;
  cfg->raster = GP_RASTER_AUTO;
  return GP_OK;
}

gp_status gp_create(gp_ctx** out, int device, const gp_config* cfg) {
  if (!out) return GP_ERR_ARG;
  *out = nullptr;
  gp_config c;
  gp_config_default(&c);
  if (cfg) {
    c = *cfg;
    if (!(c.eps > 0.0f && c.eps < 1.0f)) return GP_ERR_ARG;
    if (c.tile != 8 && c.tile != 16) return GP_ERR_ARG;
    if (c.exp_mode != GP_EXP_POLY && c.exp_mode != GP_EXP_HW && c.exp_mode != GP_EXP_POLY_ROW) return GP_ERR_ARG;
    if (c.exp_mode == GP_EXP_POLY_ROW && (c.fwd_px != 0 || c.bwd_px != 0)) return GP_ERR_ARG;
    if (c.workspace_limit < 0) return GP_ERR_ARG;
    if (c.fwd_px < 0 || (c.fwd_px > 0 && !fwd_px_supported(c.tile, c.fwd_px))) return GP_ERR_ARG;
    if (c.bwd_px < 0 || (c.bwd_px > 0 && !bwd_px_supported(c.tile, c.bwd_px))) return GP_ERR_ARG;
    if (c.raster != GP_RASTER_AUTO && c.raster != GP_RASTER_BLOCK && c.raster != GP_RASTER_ROWS) return GP_ERR_ARG;
    if (c.exp_mode == GP_EXP_POLY_ROW && c.raster == GP_RASTER_ROWS) return GP_ERR_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return GP_ERR_CUDA;
  gp_ctx* ctx = new (std::nothrow) gp_ctx();
  if (!ctx) return GP_ERR_OOM;
  ctx->impl.device = device;
  ctx->impl.cfg = c;
  if (cudaMallocHost(&ctx->impl.h_total, 64) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return GP_ERR_OOM;
  }
  if (cudaEventCreateWithFlags(&ctx->impl.bin_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->impl.scan_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->impl.side_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->impl.bin_ev) cudaEventDestroy(ctx->impl.bin_ev);
    if (ctx->impl.scan_ev) cudaEventDestroy(ctx->impl.scan_ev);
    cudaFreeHost(ctx->impl.h_total);
    delete ctx;
    return GP_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->impl.sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = ctx;
  return GP_OK;
}

gp_status gp_destroy(gp_ctx* ctx) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  ws_release_all(c);
  for (auto& e : c->events) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->h_total) cudaFreeHost(c->h_total);
  if (c->bin_ev) cudaEventDestroy(c->bin_ev);
  if (c->scan_ev) cudaEventDestroy(c->scan_ev);
  if (c->side_st) cudaStreamDestroy(c->side_st);
  delete ctx;
  return GP_OK;
}

const char* gp_last_error(gp_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->impl.err.c_str();
}

int64_t gp_workspace_bytes(gp_ctx* ctx) { return ctx ? ctx->impl.ws_bytes : 0; }

gp_status gp_last_counts(gp_ctx* ctx, int64_t* pairs, int64_t* issued) {
  if (!ctx) return GP_ERR_ARG;
  if (pairs) *pairs = ctx->impl.last_pairs;
  if (issued) *issued = ctx->impl.last_issued;
  return GP_OK;
}

static gp_status render_impl(gp_ctx* ctx, const gp_set* set, const View& view, const float* z, int S, int H,
                             int W, float sigma_z, float* out, void* stream, bool vox = false) {
  Ctx* c = &ctx->impl;
  GP_TRY(check_set(c, set));
  if (!out && S > 0) return set_err(c, GP_ERR_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  SliceArgs a;
  uint32_t P = 0;
  const uint32_t* vals = nullptr;
  // the first attempt bins speculatively; a count that overflowed the buffers
  // is binned again with its readback, and the forward repeated
  for (int attempt = 0;; ++attempt) {
    GP_TRY(bin_slices(c, set, z, S, H, W, sigma_z, view, st, &a, &P, &vals, vox, attempt == 0));
    if (S == 0) return GP_OK;
    if (P == 0) {
      GP_CUDA(c, cudaMemsetAsync(out, 0, (size_t)S * H * W * 4, st), "clear out");
      return check_after(c, st);
    }
    {
      PhaseTimer timer(c, vox ? GP_PHASE_VOX_FWD : GP_PHASE_FWD, st);
      GP_CUDA(c, launch_raster_fwd(a, fwd_px(c), c->cfg.raster, c->cfg.exp_mode, (const SliceRec*)c->b.rec.ptr, vals,
                                   c->bin_gid_vals ? nullptr : (const uint32_t*)c->b.emit_gid.ptr,
                                   (const uint2*)c->b.ranges.ptr, out, st, P),
              "raster forward");
    }
    bool redo = false;
    GP_TRY(finish_bin(c, &redo));
    if (!redo) break;
  }
  return check_after(c, st);
}

static gp_status backward_impl(gp_ctx* ctx, const gp_set* set, const View& view, const float* z, int S, int H,
                               int W, float sigma_z, const float* dL_dI, float* d_mu, float* d_scale,
                               float* d_quat, float* d_alpha, void* stream, bool vox = false) {
  Ctx* c = &ctx->impl;
  GP_TRY(check_set(c, set));
  const int n = (int)set->n;
  GP_TRY(check_grads(c, n, d_mu, d_scale, d_quat, d_alpha));
  if (S > 0 && !dL_dI) return set_err(c, GP_ERR_ARG, "dL_dI is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  SliceArgs a;
  uint32_t P = 0;
  const uint32_t* vals = nullptr;
  if (vox) sigma_z = 0.0f;  // the key of voxelizer bins (slices never have sigma_z = 0)
  const bool reuse = c->cfg.reuse_bins && S > 0 && z && bins_match(c, set, z, S, H, W, sigma_z, view);
  // a fresh binning is speculative on the first attempt (see render_impl)
  for (int attempt = 0;; ++attempt) {
    if (reuse) {
      memcpy(&a, c->bin_args, sizeof(SliceArgs));
      P = c->bin_pairs;
      vals = c->bin_vals;
    } else {
      GP_TRY(bin_slices(c, set, z, S, H, W, sigma_z, view, st, &a, &P, &vals, vox, attempt == 0));
    }
    if (n == 0) {
      bool redo = false;
      GP_TRY(finish_bin(c, &redo));
      return GP_OK;
    }
    BinBufs& b = c->b;
    GP_TRY(ws_reserve(c, b.accum, (size_t)n * 10 * 4));
    const bool det = c->cfg.deterministic != 0;
    if (det) {
      GP_TRY(ws_reserve(c, b.partial, (size_t)std::max<uint32_t>(P, 1) * 32));
    } else {
      GP_CUDA(c, cudaMemsetAsync(b.accum.ptr, 0, (size_t)n * 10 * 4, st), "clear accumulators");
    }
    if (P > 0) {
      PhaseTimer timer(c, vox ? GP_PHASE_VOX_BWD : GP_PHASE_BWD, st);
      GP_CUDA(c, launch_raster_bwd(a, bwd_px(c), c->cfg.raster, c->cfg.exp_mode, det, (const SliceRec*)b.rec.ptr,
                                   vals, c->bin_gid_vals ? nullptr : (const uint32_t*)b.emit_gid.ptr,
                                   (const uint2*)b.ranges.ptr, dL_dI,
                                   (float*)b.accum.ptr, (float4*)b.partial.ptr, st),
              "raster backward");
    }
    {
      PhaseTimer timer(c, vox ? GP_PHASE_VOX_BWD : GP_PHASE_BWD_PRE, st);
      if (det)
        // bounded by the pairs the partials hold: a speculative binning whose
        // count overflowed them is redone, but its reduce must stay in bounds
        launch_det_reduce_n(n, (const unsigned long long*)b.offsets.ptr, (const unsigned long long*)b.counts.ptr,
                            (const float4*)b.partial.ptr, (float*)b.accum.ptr, (unsigned long long)P, st);
      launch_slice_bwd_pre(a, (const float*)b.accum.ptr, d_mu, d_scale, d_quat, d_alpha, st);
    }
    GP_TRY(cuda_err(c, cudaGetLastError(), "backward kernels"));
    bool redo = false;
    GP_TRY(finish_bin(c, &redo));
    if (!redo) break;
  }
  return check_after(c, st);
}

gp_status gp_mse_grad(gp_ctx* ctx, const float* I, const float* T, const int* t_index, int S, int H, int W,
                      float* dL_dI, float* loss, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (S < 0 || H <= 0 || W <= 0) return set_err(c, GP_ERR_ARG, "need S >= 0, H > 0, W > 0");
  if (S == 0) return GP_OK;
  if (!I || !T || !dL_dI) return set_err(c, GP_ERR_ARG, "NULL image pointer");
  cudaStream_t st = (cudaStream_t)stream;
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  const int64_t HW = (int64_t)H * W;
  BinBufs& b = c->b;
  const size_t tmp_bytes = ((size_t)mse_tmp_floats(S, HW) * 4 + 255) & ~(size_t)255;
  GP_TRY(ws_reserve(c, b.loss_tmp, tmp_bytes + (size_t)S * 4));
  const int* tid = nullptr;
  if (t_index) {
    for (int s = 0; s < S; ++s)
      if (t_index[s] < 0) return set_err(c, GP_ERR_ARG, "negative target slice index");
    int* dst = (int*)((char*)b.loss_tmp.ptr + tmp_bytes);
    uint32_t* d1[1] = {(uint32_t*)dst};
    const void* s1[1] = {t_index};
    GP_CUDA(c, put_words(st, 1, d1, s1, &S), "upload t_index");
    tid = dst;
  }
  PhaseTimer timer(c, GP_PHASE_LOSS, st);
  launch_mse(I, T, tid, S, HW, dL_dI, loss, (float*)b.loss_tmp.ptr, st);
  return cuda_err(c, cudaGetLastError(), "mse");
}

// units: count the pixels the context's default rasterisers evaluate,
// evals[0] forward and evals[1] backward, instead of the algorithmic
// evaluations (evals[0]).
static gp_status count_impl(gp_ctx* ctx, const gp_set* set, const View& view, const float* z, int S, int H,
                            int W, float sigma_z, int64_t* evals, bool vox = false, bool units = false) {
  Ctx* c = &ctx->impl;
  GP_TRY(check_set(c, set));
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  cudaStream_t st = 0;
  SliceArgs a;
  uint32_t P = 0;
  const uint32_t* vals = nullptr;
  GP_TRY(bin_slices(c, set, z, S, H, W, sigma_z, view, st, &a, &P, &vals, vox));
  unsigned long long* d = (unsigned long long*)c->b.total.ptr + 1;
  GP_CUDA(c, cudaMemsetAsync(d, 0, 16, st), "count");
  if (set->n > 0 && S > 0) {
    if (units)
      launch_count_units(a, (const SliceRec*)c->b.rec.ptr, raster_rows_form(a, c->cfg.raster, c->cfg.exp_mode, false),
                         raster_rows_form(a, c->cfg.raster, c->cfg.exp_mode, true), d, st);
    else
      launch_count_evals(a, (const SliceRec*)c->b.rec.ptr, d, st);
  }
  GP_CUDA(c, cudaMemcpyAsync(c->h_total, d, 16, cudaMemcpyDeviceToHost, st), "count readback");
  GP_CUDA(c, cudaStreamSynchronize(st), "count readback");
  evals[0] = (int64_t)c->h_total[0];
  if (units) evals[1] = (int64_t)c->h_total[1];
  return GP_OK;
}

gp_status gp_view_from_axis(int axis, gp_view* view) {
  View v;
  if (!view || !axis_view(axis, &v)) return GP_ERR_ARG;
  memcpy(view->R, v.R, sizeof(v.R));
  memcpy(view->t, v.t, sizeof(v.t));
  return GP_OK;
}

gp_status gp_render_slices(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H, int W, float sigma_z,
                           int axis, float* out, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  View v;
  if (!axis_view(axis, &v)) return set_err(&ctx->impl, GP_ERR_ARG, "axis must be 0, 1 or 2");
  return render_impl(ctx, set, v, z, S, H, W, sigma_z, out, stream);
}

gp_status gp_render_slices_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z, int S,
                                int H, int W, float sigma_z, float* out, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  View v;
  if (!check_view(view, &v))
    return set_err(&ctx->impl, GP_ERR_ARG, "view must be finite with R orthonormal to 1e-3");
  return render_impl(ctx, set, v, z, S, H, W, sigma_z, out, stream);
}

gp_status gp_render_backward(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H, int W,
                             float sigma_z, int axis, const float* dL_dI, float* d_mu, float* d_scale,
                             float* d_quat, float* d_alpha, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  View v;
  if (!axis_view(axis, &v)) return set_err(&ctx->impl, GP_ERR_ARG, "axis must be 0, 1 or 2");
  return backward_impl(ctx, set, v, z, S, H, W, sigma_z, dL_dI, d_mu, d_scale, d_quat, d_alpha, stream);
}

gp_status gp_render_backward_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z, int S,
                                  int H, int W, float sigma_z, const float* dL_dI, float* d_mu, float* d_scale,
                                  float* d_quat, float* d_alpha, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  View v;
  if (!check_view(view, &v))
    return set_err(&ctx->impl, GP_ERR_ARG, "view must be finite with R orthonormal to 1e-3");
  return backward_impl(ctx, set, v, z, S, H, W, sigma_z, dL_dI, d_mu, d_scale, d_quat, d_alpha, stream);
}

gp_status gp_count_evals(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H, int W, float sigma_z,
                         int axis, int64_t* evals) {
  if (!ctx || !evals) return GP_ERR_ARG;
  View v;
  if (!axis_view(axis, &v)) return set_err(&ctx->impl, GP_ERR_ARG, "axis must be 0, 1 or 2");
  return count_impl(ctx, set, v, z, S, H, W, sigma_z, evals);
}

gp_status gp_count_evals_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z, int S,
                              int H, int W, float sigma_z, int64_t* evals) {
  if (!ctx || !evals) return GP_ERR_ARG;
  View v;
  if (!check_view(view, &v))
    return set_err(&ctx->impl, GP_ERR_ARG, "view must be finite with R orthonormal to 1e-3");
  return count_impl(ctx, set, v, z, S, H, W, sigma_z, evals);
}

gp_status gp_count_evaluated_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z, int S,
                                  int H, int W, float sigma_z, int64_t* fwd, int64_t* bwd) {
  if (!ctx || !fwd || !bwd) return GP_ERR_ARG;
  View v;
  if (!check_view(view, &v))
    return set_err(&ctx->impl, GP_ERR_ARG, "view must be finite with R orthonormal to 1e-3");
  int64_t e[2] = {0, 0};
  GP_TRY(count_impl(ctx, set, v, z, S, H, W, sigma_z, e, false, true));
  *fwd = e[0];
  *bwd = e[1];
  return GP_OK;
}

gp_status gp_exp2_eval(gp_ctx* ctx, const float* x, float* y, int64_t n, int mode, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (n < 0 || (n > 0 && (!x || !y))) return set_err(c, GP_ERR_ARG, "bad exp2 arguments");
  if (mode != GP_EXP_POLY && mode != GP_EXP_HW && mode != GP_EXP_POLY_PACKED && mode != GP_EXP_POLY_GRAD &&
      mode != GP_EXP_POLY_GRAD_PACKED)
    return set_err(c, GP_ERR_ARG, "bad exp mode");
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  launch_exp2_eval(x, y, n, mode, (cudaStream_t)stream);
  return cuda_err(c, cudaGetLastError(), "exp2 eval");
}

// The voxelizer (Eq. 12) runs as a stack of Z planes through the slice path:
// on the plane z the Gaussian is alpha exp(-delta^2 / 2 Sigma_zz) exp(-d^T
// Sigma_2d^-1 d / 2) with Sigma_2d the conditional covariance, i.e. the slice
// operator with sigma_z = 0 and amplitude alpha; voxel (ix, iy, iz) is pixel
// (ix, iy) of plane iz + 1/2, and the [Z, Y, X] volume is the [S, H, W] stack.
static gp_status vox_planes(Ctx* c, int X, int Y, int Z, std::vector<float>& z) {
  if (X <= 0 || Y <= 0 || Z <= 0) return set_err(c, GP_ERR_ARG, "need X, Y, Z > 0");
  z.resize(Z);
  for (int k = 0; k < Z; ++k) z[k] = (float)k + 0.5f;
  return GP_OK;
}

gp_status gp_voxelize(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, float* vol, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!vol) return set_err(c, GP_ERR_ARG, "vol is NULL");
  std::vector<float> z;
  GP_TRY(vox_planes(c, X, Y, Z, z));
  View v;
  axis_view(2, &v);
  return render_impl(ctx, set, v, z.data(), Z, Y, X, 0.0f, vol, stream, true);
}

gp_status gp_count_vox_evals(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, int64_t* evals) {
  if (!ctx || !evals) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  std::vector<float> z;
  GP_TRY(vox_planes(c, X, Y, Z, z));
  View v;
  axis_view(2, &v);
  return count_impl(ctx, set, v, z.data(), Z, Y, X, 0.0f, evals, true);
}

gp_status gp_count_vox_evaluated(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, int64_t* fwd, int64_t* bwd) {
  if (!ctx || !fwd || !bwd) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  std::vector<float> z;
  GP_TRY(vox_planes(c, X, Y, Z, z));
  View v;
  axis_view(2, &v);
  int64_t e[2] = {0, 0};
  GP_TRY(count_impl(ctx, set, v, z.data(), Z, Y, X, 0.0f, e, true, true));
  *fwd = e[0];
  *bwd = e[1];
  return GP_OK;
}

gp_status gp_voxelize_backward(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, const float* dL_dV,
                               float* d_mu, float* d_scale, float* d_quat, float* d_alpha, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (!dL_dV) return set_err(c, GP_ERR_ARG, "dL_dV is NULL");
  std::vector<float> z;
  GP_TRY(vox_planes(c, X, Y, Z, z));
  View v;
  axis_view(2, &v);
  return backward_impl(ctx, set, v, z.data(), Z, Y, X, 0.0f, dL_dV, d_mu, d_scale, d_quat, d_alpha, stream, true);
}

gp_status gp_timing_enable(gp_ctx* ctx, int enable) {
  if (!ctx) return GP_ERR_ARG;
  ctx->impl.timing = enable != 0 ? (1u << GP_NUM_PHASES) - 1u : 0u;
  return GP_OK;
}

gp_status gp_timing_enable_phases(gp_ctx* ctx, unsigned mask) {
  if (!ctx || (mask >> GP_NUM_PHASES) != 0u) return GP_ERR_ARG;
  ctx->impl.timing = mask;
  return GP_OK;
}

gp_status gp_timing_read(gp_ctx* ctx, double* ms, int64_t* launches, int64_t* calls) {
  if (!ctx || !ms || !launches) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  for (int k = 0; k < GP_NUM_PHASES; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    if (calls) calls[k] = 0;
  }
  gp_status st = GP_OK;
  for (auto& e : c->events) {
    float t = 0.f;
    cudaError_t r = cudaEventSynchronize(e.stop);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&t, e.start, e.stop);
    if (r != cudaSuccess) st = cuda_err(c, r, "timing event");
    if (e.phase >= 0 && e.phase < GP_NUM_PHASES) {
      ms[e.phase] += t;
      launches[e.phase] += e.launches;
      if (calls) calls[e.phase] += 1;
    }
    c->event_pool.push_back(e.start);
    c->event_pool.push_back(e.stop);
  }
  c->events.clear();
  return st;
}

int64_t gp_launch_count(void) { return launch_count(); }

int64_t gp_fma_probe_threads(gp_ctx* ctx) { return ctx ? fma_probe_threads(ctx->impl.sm_count) : 0; }

gp_status gp_fma_probe_mode(gp_ctx* ctx, int mode, int iters, float* out, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
  if (iters <= 0 || !out || mode < 0 || mode > 3) return set_err(c, GP_ERR_ARG, "bad probe arguments");
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  launch_fma_probe(c->sm_count, mode, iters, out, (cudaStream_t)stream);
  return cuda_err(c, cudaGetLastError(), "fma probe");
}

gp_status gp_fma_probe(gp_ctx* ctx, int iters, float* out, void* stream) {
  return gp_fma_probe_mode(ctx, 0, iters, out, stream);
}

int gp_fma_probe_lane_fmas(int mode) { return (mode >= 0 && mode <= 3) ? fma_probe_lane_fmas(mode) : 0; }

int gp_check_enabled(void) {
#ifdef GP_CHECK
  return 1;
#else
  return 0;
#endif
}

gp_status gp_check_selftest(gp_ctx* ctx, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  Ctx* c = &ctx->impl;
#ifdef GP_CHECK
  GP_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  launch_check_selftest((cudaStream_t)stream);
  GP_CUDA(c, cudaGetLastError(), "check selftest");
  return check_after(c, (cudaStream_t)stream);
#else
  (void)stream;
  return set_err(c, GP_ERR_STATE, "not a bounds-checked build");
#endif
}

}  // extern "C"
