// sort.cu -- device-wide exclusive scan and a stable LSD radix sort of 32-bit
// (slice, tile) keys with 32-bit values, written for sm_103a.
//
// The renderer's binning (the "binned to screen tiles" step of the operator)
// needs the Gaussians of every (slice, tile) contiguous and, inside a tile, in
// ascending emission (= Gaussian id) order so that sums are reproducible.  Keys
// are emitted in that order, so a STABLE sort on the key alone suffices.  The
// values carried along are the identity (emission indices) or the caller's
// first-pass values (the Gaussian ids).
//
// Radix sort, per 8-bit digit pass:
//   1. k_radix_hist     per 4096-key tile: 256-bin histogram (shared atomics),
//                       stored digit-major hist[d * nb + b];
//   2. k_radix_colscan  one CTA per digit: exclusive scan of the digit's row
//                       over the tiles (in place) and the digit's total;
//   3. k_radix_scatter  per tile: the digits' global starts (a scan of the 256
//                       totals plus the tile's row entry); each warp ranks its own 512 keys in 16 rounds
//                       of 32 (nine ballots give each key the lanes holding the
//                       same digit, a running per-warp digit count the rest), a
//                       per-digit prefix over the 8 warps gives tile-local
//                       positions -> a stable local sort in shared memory, then
//                       each digit's run is stored contiguously.
// Only ceil(bits / 8) passes run; bits is the number of live key bits.
// Counts are read from device memory (n_dev) with a host-side capacity bound on
// the grid, so the same launches serve a preplanned (graph-captured) binning.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "gp_check.cuh"
#include "gp_internal.h"

namespace gp {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of the block's per-thread values; returns the thread's prefix
// and writes the block total to *total.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem_warp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) smem_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NT / 32 ? smem_warp[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < NT / 32) smem_warp[lane] = wi - w;
    if (lane == NT / 32 - 1) smem_warp[NT / 32] = wi;
  }
  __syncthreads();
  T r = smem_warp[warp] + inc - v;
  *total = smem_warp[NT / 32];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const T* __restrict__ in, int64_t n,
                                                               unsigned long long* __restrict__ part) {
  __shared__ unsigned long long sw[SCAN_THREADS / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (unsigned long long)in[i];
  }
  unsigned long long tot;
  block_exclusive_scan<unsigned long long, SCAN_THREADS>(s, sw, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// One block scans the per-tile partials (exclusive) and writes the grand total.
__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* __restrict__ part, int nb,
                                                        unsigned long long* __restrict__ total) {
  __shared__ unsigned long long sw[1024 / 32 + 1];
  unsigned long long carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    unsigned long long v = i < nb ? part[i] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan<unsigned long long, 1024>(v, sw, &tot);
    if (i < nb) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// The SCAN_ITEMS consecutive items of one thread (blocked arrangement): as
// 16-byte loads / stores when they are all in range and the address is
// 16-byte aligned, item by item otherwise.
template <typename T>
__device__ __forceinline__ void load_items(const T* __restrict__ in, int64_t base, int64_t n, T (&v)[SCAN_ITEMS]) {
  static_assert((SCAN_ITEMS * sizeof(T)) % 16 == 0, "whole 16-byte vectors");
  if (base + SCAN_ITEMS <= n && (reinterpret_cast<uintptr_t>(in + base) & 15u) == 0) {
    uint4 w[SCAN_ITEMS * sizeof(T) / 16];
#pragma unroll
    for (int k = 0; k < (int)(SCAN_ITEMS * sizeof(T) / 16); ++k) w[k] = reinterpret_cast<const uint4*>(in + base)[k];
    memcpy(v, w, sizeof(w));
    return;
  }
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = base + k < n ? in[base + k] : T(0);
}

template <typename T>
__device__ __forceinline__ void store_items(T* __restrict__ out, int64_t base, int64_t n, const T (&v)[SCAN_ITEMS]) {
  if (base + SCAN_ITEMS <= n && (reinterpret_cast<uintptr_t>(out + base) & 15u) == 0) {
    uint4 w[SCAN_ITEMS * sizeof(T) / 16];
    memcpy(w, v, sizeof(w));
#pragma unroll
    for (int k = 0; k < (int)(SCAN_ITEMS * sizeof(T) / 16); ++k) reinterpret_cast<uint4*>(out + base)[k] = w[k];
    return;
  }
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) out[base + k] = v[k];
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const T* __restrict__ in, T* __restrict__ out,
                                                             int64_t n,
                                                             const unsigned long long* __restrict__ part) {
  __shared__ unsigned long long sw[SCAN_THREADS / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  unsigned long long s = 0;
  // blocked arrangement: thread t owns SCAN_ITEMS consecutive items
  load_items(in, base, n, v);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) s += (unsigned long long)v[k];
  unsigned long long tot;
  unsigned long long ex = block_exclusive_scan<unsigned long long, SCAN_THREADS>(s, sw, &tot);
  unsigned long long run = part[blockIdx.x] + ex;
  T o[SCAN_ITEMS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    o[k] = (T)run;
    run += (unsigned long long)v[k];
  }
  store_items(out, base, n, o);
}

int64_t scan_temp_bytes(int64_t n) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (nb + 1) * (int64_t)sizeof(unsigned long long);
}

// Short arrays (up to SCAN_SMALL_TILES tiles) in one launch: every block first
// sums all the items before its tile (coalesced; the redundant reads are a few
// tiles at most), then scans its own tile as k_scan_down does.
constexpr int SCAN_SMALL_TILES = 8;

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_small(const T* __restrict__ in, T* __restrict__ out,
                                                              int64_t n, unsigned long long* __restrict__ total) {
  __shared__ unsigned long long sw[SCAN_THREADS / 32 + 1];
  const int64_t tile0 = (int64_t)blockIdx.x * SCAN_TILE;
  unsigned long long c = 0;
  for (int64_t i = threadIdx.x; i < tile0; i += SCAN_THREADS) c += (unsigned long long)in[i];
  unsigned long long carry;
  block_exclusive_scan<unsigned long long, SCAN_THREADS>(c, sw, &carry);
  const int64_t base = tile0 + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  unsigned long long s = 0;
  load_items(in, base, n, v);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) s += (unsigned long long)v[k];
  unsigned long long tot;
  unsigned long long run = carry + block_exclusive_scan<unsigned long long, SCAN_THREADS>(s, sw, &tot);
  T o[SCAN_ITEMS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    o[k] = (T)run;
    run += (unsigned long long)v[k];
  }
  store_items(out, base, n, o);
  if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = carry + tot;
}

template <typename T>
cudaError_t exclusive_scan(const T* in, T* out, int64_t n, unsigned long long* total, void* temp,
                           cudaStream_t st) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned long long* part = (unsigned long long*)temp;
  if (nb == 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
    return cudaSuccess;
  }
  if (nb <= SCAN_SMALL_TILES) {
    k_scan_small<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, total);
    note_launch();
    return cudaGetLastError();
  }
  k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, part);
  k_scan_partials<<<1, 1024, 0, st>>>(part, (int)nb, total);
  k_scan_down<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, part);
  note_launch(3);
  return cudaGetLastError();
}

template cudaError_t exclusive_scan<uint32_t>(const uint32_t*, uint32_t*, int64_t, unsigned long long*,
                                              void*, cudaStream_t);
template cudaError_t exclusive_scan<unsigned long long>(const unsigned long long*, unsigned long long*,
                                                        int64_t, unsigned long long*, void*, cudaStream_t);

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

__device__ __forceinline__ uint32_t load_count(const unsigned long long* n_dev, uint32_t cap) {
  unsigned long long n = *n_dev;
  return n < cap ? (uint32_t)n : cap;
}

// Keys are read as 16-byte vectors, all four loads of a thread issued before
// its shared-memory atomics (the tile's first key is a multiple of 4096, so
// with a 16-byte aligned key array every vector is aligned; a vector that
// would run past cap is read key by key).
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ keys,
                                                            const unsigned long long* __restrict__ n_dev,
                                                            uint32_t cap, int shift,
                                                            uint32_t* __restrict__ hist, int nb) {
  __shared__ uint32_t cnt[RS_BINS];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t n = load_count(n_dev, cap);
  uint32_t base = blockIdx.x * RS_TILE;
  if (base < n) {
    constexpr int NV = RS_ROUNDS / 4;  // 16-byte vectors per thread
    uint4 v[NV];
#pragma unroll
    for (int r = 0; r < NV; ++r) {
      const uint32_t i = base + 4u * (uint32_t)(r * RS_THREADS + threadIdx.x);
      if (i + 4u <= cap) {
        v[r] = *reinterpret_cast<const uint4*>(keys + i);
      } else {
        v[r].x = i < cap ? keys[i] : 0u;
        v[r].y = i + 1u < cap ? keys[i + 1u] : 0u;
        v[r].z = i + 2u < cap ? keys[i + 2u] : 0u;
        v[r].w = i + 3u < cap ? keys[i + 3u] : 0u;
      }
    }
#pragma unroll
    for (int r = 0; r < NV; ++r) {
      const uint32_t i = base + 4u * (uint32_t)(r * RS_THREADS + threadIdx.x);
      const uint32_t k4[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i + (uint32_t)q < n) atomicAdd(&cnt[(k4[q] >> shift) & 0xffu], 1u);
    }
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of each digit's row of the digit-major histogram over the
// tiles, in place, one CTA per digit, and the digit's total.
constexpr int CS_THREADS = 512;
constexpr int CS_ITEMS = 8;

__global__ void __launch_bounds__(CS_THREADS) k_radix_colscan(uint32_t* __restrict__ hist, int nb,
                                                               uint32_t* __restrict__ dtot) {
  __shared__ uint32_t sw[CS_THREADS / 32 + 1];
  uint32_t* row = hist + (size_t)blockIdx.x * nb;
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += CS_THREADS * CS_ITEMS) {
    const int i0 = base + threadIdx.x * CS_ITEMS;
    uint32_t v[CS_ITEMS], sum = 0;
#pragma unroll
    for (int k = 0; k < CS_ITEMS; ++k) {
      v[k] = i0 + k < nb ? row[i0 + k] : 0u;
      sum += v[k];
    }
    uint32_t tot;
    uint32_t run = carry + block_exclusive_scan<uint32_t, CS_THREADS>(sum, sw, &tot);
#pragma unroll
    for (int k = 0; k < CS_ITEMS; ++k) {
      if (i0 + k < nb) row[i0 + k] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

// Stable scatter of one 4096-key tile.  Warp w owns the tile's keys
// [w * 512, (w + 1) * 512) and ranks them in 16 rounds of 32 against its own
// per-digit counters (nine ballots give the rank among equal digits in a round),
// keeping key, value and rank in registers.  A block-wide pass turns the
// per-warp counts into tile-local digit offsets; the keys are first placed in
// shared memory in digit order (a stable local sort), and then written out in
// that order, so each digit's run leaves the block as contiguous stores.
constexpr int RS_PER_WARP = RS_TILE / RS_WARPS;     // 512 keys
constexpr int RS_ROUNDS_W = RS_PER_WARP / 32;       // 16 rounds

__global__ void __launch_bounds__(RS_THREADS, 3) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const unsigned long long* __restrict__ n_dev, uint32_t cap, int shift,
    const uint32_t* __restrict__ hist, int nb, const uint32_t* __restrict__ dtot) {
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t dlocal[RS_BINS];   // tile-local start of each digit
  __shared__ uint32_t dglobal[RS_BINS];  // global start of each digit of this tile
  __shared__ uint32_t skey[RS_TILE], sval[RS_TILE];
  __shared__ uint32_t swarp[RS_WARPS + 1], sgw[RS_WARPS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t n = load_count(n_dev, cap);
  const uint32_t tile0 = blockIdx.x * RS_TILE;
  if (tile0 >= n) return;  // uniform across the block
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wcnt[w][t] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t base = tile0 + warp * RS_PER_WARP;
  uint32_t key[RS_ROUNDS_W], val[RS_ROUNDS_W], rank[RS_ROUNDS_W];
  // every load of the thread first (keys and values, held in registers: 3 CTAs
  // per SM with 80 registers beat 4 with the values read at the placement): the
  // ranking rounds below are separated by __syncwarp, which would otherwise
  // hold each round's load back until the previous round is done
#pragma unroll
  for (int r = 0; r < RS_ROUNDS_W; ++r) {
    const uint32_t i = base + r * 32 + lane;
    key[r] = i < n ? kin[i] : 0u;
    val[r] = i < n ? (vin ? vin[i] : i) : 0u;  // no input values: the identity
  }
  // NB = 8 on a tile whose keys are all valid; NB = 9 on the last, partial
  // tile, where the ninth ballot sets the invalid lanes apart
  auto rank_keys = [&](auto nb_tag) {
    constexpr int NB = decltype(nb_tag)::value;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS_W; ++r) {
      const uint32_t i = base + r * 32 + lane;
      const bool valid = NB == 8 || i < n;
      const uint32_t d = valid ? ((key[r] >> shift) & 0xffu) : (RS_BINS + lane);
      // lanes holding the same digit: one ballot per digit bit (and one for
      // validity; an invalid lane's low bits are its lane number, so it is alone)
      uint32_t peers = 0xffffffffu;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
      }
      uint32_t c = 0u;
      if (valid) c = wcnt[warp][d];
      rank[r] = valid ? c + __popc(peers & lt_mask) : 0xffffffffu;
      __syncwarp();
      if (valid && __popc(peers & lt_mask) == 0) wcnt[warp][d] = c + __popc(peers);
      __syncwarp();
    }
  };
  if (tile0 + (uint32_t)RS_TILE <= n)  // uniform across the block
    rank_keys(std::integral_constant<int, 8>{});
  else
    rank_keys(std::integral_constant<int, 9>{});
  __syncthreads();
  // thread t owns digit t: per-warp offsets inside the digit, the digit's tile total
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    const uint32_t c = wcnt[w][t];
    wcnt[w][t] = tot;
    tot += c;
  }
  // exclusive scans over the 256 digits (warp scans + warp sums): the tile's
  // digit totals (tile-local starts) and the digits' totals over all keys
  // (where each digit starts in the output)
  const uint32_t g = dtot[t];
  uint32_t inc = tot, ginc = g;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    const uint32_t gu = __shfl_up_sync(0xffffffffu, ginc, o);
    if (lane >= o) {
      inc += u;
      ginc += gu;
    }
  }
  if (lane == 31) {
    swarp[warp] = inc;
    sgw[warp] = ginc;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0, grun = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = swarp[w], gc = sgw[w];
      swarp[w] = run;
      sgw[w] = grun;
      run += c;
      grun += gc;
    }
    swarp[RS_WARPS] = run;
  }
  __syncthreads();
  dlocal[t] = swarp[warp] + inc - tot;
  dglobal[t] = sgw[warp] + ginc - g + hist[(size_t)t * nb + blockIdx.x];
  __syncthreads();
  // local stable placement in digit order
#pragma unroll
  for (int r = 0; r < RS_ROUNDS_W; ++r) {
    if (rank[r] != 0xffffffffu) {
      const uint32_t d = (key[r] >> shift) & 0xffu;
      const uint32_t lp = dlocal[d] + wcnt[warp][d] + rank[r];
      if (GP_IN_RANGE(11, lp, RS_TILE)) {
        skey[lp] = key[r];
        sval[lp] = val[r];
      }
    }
  }
  __syncthreads();
  const uint32_t count = swarp[RS_WARPS];
  for (uint32_t lp = t; lp < count; lp += RS_THREADS) {
    const uint32_t k = skey[lp];
    const uint32_t d = (k >> shift) & 0xffu;
    const uint32_t pos = dglobal[d] + (lp - dlocal[d]);
    if (GP_IN_RANGE(10, pos, n)) {
      kout[pos] = k;
      vout[pos] = sval[lp];
    }
  }
}

int64_t radix_temp_bytes(int64_t cap) {
  int64_t nb = (cap + RS_TILE - 1) / RS_TILE;
  int64_t hist = (int64_t)RS_BINS * nb;
  return ((hist * 4 + 255) / 256) * 256 + RS_BINS * 4;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                             const unsigned long long* n_dev, uint32_t cap, int bits, void* temp,
                             cudaStream_t st, bool* result_in_alt, const uint32_t* first_vals) {
  *result_in_alt = false;
  if (cap == 0 || bits <= 0) return cudaSuccess;
  if ((((uintptr_t)keys) | ((uintptr_t)keys_alt)) & 15u) return cudaErrorMisalignedAddress;
  int nb = (int)((cap + RS_TILE - 1) / RS_TILE);
  uint32_t* hist = (uint32_t*)temp;
  int64_t nh = (int64_t)RS_BINS * nb;
  uint32_t* dtot = (uint32_t*)((char*)temp + ((nh * 4 + 255) / 256) * 256);
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<nb, RS_THREADS, 0, st>>>(ki, n_dev, cap, shift, hist, nb);
    k_radix_colscan<<<RS_BINS, CS_THREADS, 0, st>>>(hist, nb, dtot);
    k_radix_scatter<<<nb, RS_THREADS, 0, st>>>(ki, shift == 0 ? first_vals : vi, ko, vo, n_dev, cap, shift, hist, nb,
                                               dtot);
    note_launch(3);
    uint32_t* tk = ki; ki = ko; ko = tk;
    uint32_t* tv = vi; vi = vo; vo = tv;
    *result_in_alt = !*result_in_alt;
  }
  return cudaGetLastError();
}

GP_CHECK_READER(check_read_sort)

}  // namespace gp
