// gp_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gp.h"

namespace gp {

// ------------------------------------------------------------- primitives
int64_t scan_temp_bytes(int64_t n);
template <typename T>
cudaError_t exclusive_scan(const T* in, T* out, int64_t n, unsigned long long* total, void* temp,
                           cudaStream_t st);
int64_t radix_temp_bytes(int64_t cap);
// The first pass takes first_vals as input values, or the identity 0..n-1 when
// it is NULL (vals is not read); later passes ping-pong between vals and
// vals_alt.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                             const unsigned long long* n_dev, uint32_t cap, int bits, void* temp,
                             cudaStream_t st, bool* result_in_alt, const uint32_t* first_vals = nullptr);

// Copies up to three small host arrays of 32-bit words to the device in stream
// order.  Up to 720 words in all travel as the arguments of one kernel launch
// (no copy-engine operation, no staging of pageable memory); larger arrays go
// by cudaMemcpyAsync.
cudaError_t put_words(cudaStream_t st, int k, uint32_t* const* dst, const void* const* src, const int* n);

// --------------------------------------------------------------- workspace
// A grow-only device buffer.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Ctx;

// Ensures buf holds at least `bytes`; grows by 1.25x.  Returns GP_OK or GP_ERR_OOM.
gp_status ws_reserve(Ctx* c, DevBuf& buf, size_t bytes);
void ws_release(Ctx* c, DevBuf& buf);
void ws_release_all(Ctx* c);

// Buffers of one binned render (slice renderer or voxelizer).
struct BinBufs {
  DevBuf rec;        // per-Gaussian record (64 B)
  DevBuf counts;     // per-Gaussian pair count (uint64)
  DevBuf offsets;    // exclusive scan of counts (uint64), written by K-emit
  DevBuf wsum, woff; // per warp of 32 Gaussians: pair total and its exclusive scan (uint64)
  DevBuf total;      // pair total (uint64) + spare slots
  DevBuf keys, vals, keys_alt, vals_alt;  // uint32
  DevBuf emit_gid;   // emission index -> Gaussian id (uint32)
  DevBuf ranges;     // per (slice, tile): [start, end) (uint2)
  DevBuf scan_tmp, sort_tmp;
  DevBuf zs, zorder, zorig;  // sorted plane positions, their slice indices, positions by index
  DevBuf accum;      // backward: per-Gaussian accumulators
  DevBuf partial;    // backward, deterministic mode: per-pair partials
  DevBuf loss_tmp;
  DevBuf codec;      // encode / decode scratch
};

// Adds k to the process-wide count of kernels this library launched.
void note_launch(int k = 1);
int64_t launch_count();
int64_t fma_probe_threads(int sm_count);
int fma_probe_lane_fmas(int mode);
void launch_fma_probe(int sm_count, int mode, int iters, float* out, cudaStream_t st);

struct PhaseEvent {
  int phase;
  cudaEvent_t start, stop;
  int64_t launches;
};

// A validated slice orientation [R_c | t] (camera x_c = R_c x + t, row-major R_c).
struct View {
  float R[9];
  float t[3];
};
// The permutation view of slice axis 0, 1 or 2 (false for any other axis).
bool axis_view(int axis, View* v);
// Copies a caller's view if it is finite and R is orthonormal to within 1e-3.
bool check_view(const gp_view* in, View* out);
bool same_view(const View& a, const View& b);

// Arguments of the binning currently held in a context's buffers.
struct BinKey {
  bool valid = false;
  const float *mu = nullptr, *scale = nullptr, *quat = nullptr, *alpha = nullptr;
  int64_t n = 0;
  float mod = 0.f, sigma_z = 0.f;
  std::vector<float> z;
  View view{};
  int S = 0, H = 0, W = 0, tile = 0;
};

struct Ctx {
  int device = 0;
  BinKey bin_key;          // what b.rec / b.ranges / the sorted values describe
  uint32_t bin_pairs = 0;
  const uint32_t* bin_vals = nullptr;
  bool bin_gid_vals = false;  // the sorted values are Gaussian ids (else emission indices)
  char bin_args[256];      // the SliceArgs of that binning (opaque here)
  unsigned timing = 0u;     // phases (bit GP_PHASE_*) whose calls record event pairs
  std::vector<PhaseEvent> events;
  std::vector<cudaEvent_t> event_pool;
  gp_config cfg{};
  std::string err;
  int64_t ws_bytes = 0;
  BinBufs b;
  unsigned long long* h_total = nullptr;  // pinned readback slot
  int64_t last_pairs = 0, last_issued = 0;
  // Speculative binning: the pairs were emitted and sorted into the buffers'
  // capacity (bin_cap pairs) before their count came back.  The count's copy
  // to h_total runs on side_st after scan_ev (the scan's end); bin_ev follows
  // it, and the call checks it once its rasteriser is queued.
  bool bin_pending = false;
  uint32_t bin_cap = 0;
  cudaEvent_t bin_ev = nullptr, scan_ev = nullptr;
  cudaStream_t side_st = nullptr;
  int sm_count = 148;
};

gp_status set_err(Ctx* c, gp_status st, const std::string& msg);

// Bounds-checked build (-DGP_CHECK): the first failed index check of each
// translation unit, read and cleared ((site << 40) | index, 0 = none), and a
// kernel that fails one check on purpose (it touches no memory).
#ifdef GP_CHECK
unsigned long long check_read_raster();
unsigned long long check_read_slice();
unsigned long long check_read_sort();
void launch_check_selftest(cudaStream_t st);
#endif
// In the bounds-checked build: waits for st and returns GP_ERR_STATE, naming
// the file, site and index, if a kernel skipped an out-of-range access.
// GP_OK otherwise, and always in the default build (no wait).
gp_status check_after(Ctx* c, cudaStream_t st);

// A named NVTX range on the calling host thread for the object's lifetime (a
// no-op unless a profiler is attached), so the phases of every call show up on
// an nsys / ncu timeline.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Records an event pair around a phase on stream st when timing is enabled,
// inside an NVTX range named after the phase.
class PhaseTimer {
 public:
  PhaseTimer(Ctx* c, int phase, cudaStream_t st);
  ~PhaseTimer();

 private:
  NvtxRange range_;
  Ctx* c_;
  int phase_;
  cudaStream_t st_;
  cudaEvent_t start_ = nullptr;
  int64_t l0_ = 0;
};
gp_status cuda_err(Ctx* c, cudaError_t e, const char* where);

}  // namespace gp

struct gp_ctx {
  gp::Ctx impl;
};
