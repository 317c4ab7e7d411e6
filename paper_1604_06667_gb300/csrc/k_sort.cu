// k_sort.cu -- stable least-significant-digit radix sort of (key, value) pairs.
//
// Replaces the paper's STL hash tables (Sect. 3.4: input->output and
// output->input mappings) with one sort of the samples by HEALPix RING index.
// Stability (ties keep ascending value order) makes the result a pure function
// of the input, so the gridded sums have a deterministic order.
//
// Per 8-bit digit pass:
//   k_hist     per-block digit histograms, stored digit-major, plus totals;
//   k_scan     one CTA per digit: exclusive scan of that digit's block counts,
//              offset by the count of all smaller digits;
//   k_scatter  each block ranks its keys stably (round by round, warp-level
//              match for equal digits, warps in order) and writes them out.
#include <algorithm>

#include "cg_common.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTileKeys = kThreads * kItems;
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;

template <typename K>
__global__ void __launch_bounds__(kThreads) k_hist(const K* __restrict__ keys, int64_t n,
                                                   int shift, uint32_t* __restrict__ hist,
                                                   uint32_t* __restrict__ totals, int nblk) {
  __shared__ uint32_t cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTileKeys;
#pragma unroll 4
  for (int it = 0; it < kItems; ++it) {
    const int64_t i = base + (int64_t)it * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  const uint32_t c = cnt[threadIdx.x];
  hist[(size_t)threadIdx.x * nblk + blockIdx.x] = c;
  if (c) atomicAdd(&totals[threadIdx.x], c);
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums,
                                                         uint32_t& block_total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = (lane < kWarps) ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kWarps) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t wbase = (wid > 0) ? warp_sums[wid - 1] : 0u;
  block_total = warp_sums[kWarps - 1];
  __syncthreads();
  return wbase + incl - x;
}

// One CTA per digit d: hist[d][b] <- sum(totals[0..d)) + sum_{b' < b} hist[d][b'].
__global__ void __launch_bounds__(kThreads) k_scan(uint32_t* __restrict__ hist,
                                                   const uint32_t* __restrict__ totals,
                                                   int nblk) {
  __shared__ uint32_t warp_sums[kWarps];
  __shared__ uint32_t base_s;
  const int d = blockIdx.x;
  if (threadIdx.x == 0) {
    uint32_t b = 0;
    for (int i = 0; i < d; ++i) b += totals[i];
    base_s = b;
  }
  __syncthreads();
  uint32_t carry = base_s;
  uint32_t* row = hist + (size_t)d * nblk;
  constexpr int kPer = 4;
  for (int64_t t0 = 0; t0 < nblk; t0 += (int64_t)kThreads * kPer) {
    uint32_t v[kPer];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int64_t i = t0 + (int64_t)threadIdx.x * kPer + j;
      v[j] = (i < nblk) ? row[i] : 0u;
      s += v[j];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(s, warp_sums, tot);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int64_t i = t0 + (int64_t)threadIdx.x * kPer + j;
      if (i < nblk) row[i] = carry + ex;
      ex += v[j];
    }
    carry += tot;
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_scatter(const K* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout,
                                                      uint32_t* __restrict__ vout, int64_t n,
                                                      int shift,
                                                      const uint32_t* __restrict__ offs,
                                                      int nblk) {
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t run[kRadix];
  __shared__ uint32_t gbase[kRadix];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  run[tid] = 0;
  gbase[tid] = offs[(size_t)tid * nblk + blockIdx.x];
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kTileKeys;
  for (int it = 0; it < kItems; ++it) {
    const int64_t i = base + (int64_t)it * kThreads + tid;
    const bool valid = i < n;
    K key = 0;
    uint32_t v = 0;
    unsigned d = kRadix;  // invalid lanes form their own group
    if (valid) {
      key = kin[i];
      v = vin[i];
      d = (unsigned)(key >> shift) & 0xffu;
    }
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t r = run[tid];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = r;
        r += c;
      }
      run[tid] = r;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = gbase[d] + wcnt[wid][d] + rank;
      kout[pos] = key;
      vout[pos] = v;
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t ensure_work(SortWork& w, int64_t n, int nblk, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (w.cap_n < (size_t)n || w.key_bytes != sizeof(K)) {
    if (w.keys_alt) cudaFreeAsync(w.keys_alt, s);
    dfree(w.vals_alt, s);
    w.keys_alt = nullptr;
    w.cap_n = 0;
    e = cudaMallocAsync(&w.keys_alt, (size_t)n * sizeof(K), s);
    if (e != cudaSuccess) return e;
    e = dalloc(&w.vals_alt, (size_t)n, s);
    if (e != cudaSuccess) return e;
    w.cap_n = (size_t)n;
    w.key_bytes = sizeof(K);
  }
  if (w.cap_hist < (size_t)kRadix * nblk || !w.totals) {
    dfree(w.hist, s);
    dfree(w.totals, s);
    w.cap_hist = 0;
    e = dalloc(&w.hist, (size_t)kRadix * nblk, s);
    if (e != cudaSuccess) return e;
    e = dalloc(&w.totals, (size_t)kRadix, s);
    if (e != cudaSuccess) return e;
    w.cap_hist = (size_t)kRadix * nblk;
  }
  return cudaSuccess;
}

template <typename K>
cudaError_t radix_sort_impl(K* keys, uint32_t* vals, int64_t n, int key_bits, SortWork& w,
                            cudaStream_t s, K** out_k, uint32_t** out_v) {
  *out_k = keys;
  *out_v = vals;
  if (n <= 0) return cudaSuccess;
  const int nblk = (int)ceil_div(n, kTileKeys);
  cudaError_t e = ensure_work<K>(w, n, nblk, s);
  if (e != cudaSuccess) return e;
  K* kin = keys;
  K* kout = static_cast<K*>(w.keys_alt);
  uint32_t* vin = vals;
  uint32_t* vout = w.vals_alt;
  for (int shift = 0; shift < key_bits; shift += 8) {
    e = cudaMemsetAsync(w.totals, 0, kRadix * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_hist<K><<<nblk, kThreads, 0, s>>>(kin, n, shift, w.hist, w.totals, nblk);
    k_scan<<<kRadix, kThreads, 0, s>>>(w.hist, w.totals, nblk);
    k_scatter<K><<<nblk, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, w.hist, nblk);
    K* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
  *out_k = kin;
  *out_v = vin;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-sweep passes (32-bit keys): a tile's digit offsets come from the global
// digit totals (order-independent, one histogram kernel for every pass) plus
// the counts of the tiles before it, found by decoupled look-back: each tile
// publishes its per-digit count, then its inclusive prefix, in one 64-bit
// status word per (tile, digit) tagged with the sort's epoch (no clearing
// between sorts).  Tiles take tickets in launch order, so a tile only waits
// for tiles that already run; every wait is bounded and records an error.
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 4;
constexpr uint64_t kAgg = 1, kInc = 2;
constexpr int kOsItems = 16;                      // keys per thread of a one-sweep tile
constexpr int kOsTile = kThreads * kOsItems;

__global__ void __launch_bounds__(kThreads) k_os_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                     int npass, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kMaxPasses][kRadix];
  for (int p = 0; p < kMaxPasses; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
    const uint32_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int p = 0; p < npass; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&ghist[p * kRadix + threadIdx.x], h[p][threadIdx.x]);
}

__device__ __forceinline__ uint64_t os_word(uint32_t epoch, uint64_t kind, uint32_t v) {
  return ((uint64_t)epoch << 34) | (kind << 32) | v;
}

// One pass.  Warp w of the tile ranks the keys [512 w, 512 w + 512) of the
// tile, 32 consecutive keys per round: equal digits of a round are grouped by
// a warp match, the warp's running count per digit lives in its own row of
// shared counters, so ranking needs no block barrier.  Then one block step
// turns the per-warp counts into per-warp digit offsets and the tile's digit
// counts, the look-back finds the tile's offsets, and every key is written
// to  tile offset + offset of its warp + its rank within the warp  -- the
// position of the key among equal digits follows its input position (stable).
__global__ void __launch_bounds__(kThreads) k_os_pass_warp(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
    const uint32_t* __restrict__ ghist, uint64_t* status, uint32_t* ticket, uint32_t epoch,
    unsigned* err) {
  constexpr int kPerWarp = kOsTile / kWarps;       // 512 keys per warp
  __shared__ uint32_t s_b;
  __shared__ uint32_t blk_off[kRadix];
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t warp_sums[kWarps];
  __shared__ uint32_t t_start[kRadix];      // the tile's keys before digit d
  __shared__ uint32_t s_key[kOsTile];       // the tile in sorted order
  __shared__ uint32_t s_val[kOsTile];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_b = atomicAdd(ticket, 1u);
#pragma unroll
  for (int w2 = 0; w2 < kWarps; ++w2) wcnt[w2][tid] = 0;
  __syncthreads();
  const int64_t b = s_b;
  const int64_t wbase = b * kOsTile + (int64_t)wid * kPerWarp;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t k_it[kOsItems], v_it[kOsItems], r_it[kOsItems];
#pragma unroll
  for (int it = 0; it < kOsItems; ++it) {
    const int64_t i = wbase + it * 32 + lane;
    k_it[it] = 0;
    v_it[it] = 0;
    if (i < n) {
      k_it[it] = kin[i];
      v_it[it] = vin[i];
    }
  }
  // ranks within the warp, round by round
  uint32_t* wc = wcnt[wid];
#pragma unroll
  for (int it = 0; it < kOsItems; ++it) {
    const bool valid = wbase + it * 32 + lane < n;
    const unsigned d = valid ? ((k_it[it] >> shift) & 0xffu) : (unsigned)kRadix;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt_mask);
    const uint32_t c0 = valid ? wc[d] : 0u;
    r_it[it] = c0 + before;
    __syncwarp();
    if (valid && before == 0) wc[d] = c0 + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // digit tid: offsets of the warps within the tile, and the tile's count
  uint32_t c = 0;
#pragma unroll
  for (int w2 = 0; w2 < kWarps; ++w2) {
    const uint32_t x = wcnt[w2][tid];
    wcnt[w2][tid] = c;
    c += x;
  }
  // global exclusive offset of digit tid, and the tile's own
  uint32_t tot;
  const uint32_t g_excl = block_exclusive_scan(ghist[tid], warp_sums, tot);
  t_start[tid] = block_exclusive_scan(c, warp_sums, tot);
  // publish the count, look back for the prefix, publish the prefix
  volatile uint64_t* st = status;
  if (b == 0) {
    st[(size_t)tid] = os_word(epoch, kInc, c);
    blk_off[tid] = g_excl;
  } else {
    st[(size_t)b * kRadix + tid] = os_word(epoch, kAgg, c);
    // look back 8 predecessors per step (independent loads), summing in order
    // until an inclusive prefix; a predecessor not yet published is re-read
    uint32_t prefix = 0;
    int64_t j = b - 1;
    uint32_t spins = 0;
    const long long t0 = clock64();
    bool done = false;
    while (j >= 0 && !done) {
      uint64_t wv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) wv[q] = (j - q >= 0) ? st[(size_t)(j - q) * kRadix + tid] : 0;
      int q = 0;
      for (; q < 8 && j - q >= 0; ++q) {
        const uint64_t w = wv[q];
        const uint64_t kind = (w >> 32) & 3u;
        if ((uint32_t)(w >> 34) != epoch || kind == 0) break;   // not ready yet
        prefix += (uint32_t)w;
        if (kind == kInc) {
          done = true;
          break;
        }
      }
      if (done) break;
      j -= q;
      if (q < 8 && j >= 0) {
        // never expected to take long: give up after ~1 s and record it
        if ((++spins & 63u) == 0 && clock64() - t0 > 2000000000LL) {
          set_error(err, ERR_TIMEOUT);
          break;
        }
      }
    }
    st[(size_t)b * kRadix + tid] = os_word(epoch, kInc, prefix + c);
    blk_off[tid] = g_excl + prefix;
  }
  // the tile in sorted order in shared memory, then written out in runs per
  // digit (consecutive threads, consecutive positions)
#pragma unroll
  for (int it = 0; it < kOsItems; ++it) {
    if (wbase + it * 32 + lane < n) {
      const unsigned d = (k_it[it] >> shift) & 0xffu;
      const uint32_t lp = t_start[d] + wc[d] + r_it[it];
      s_key[lp] = k_it[it];
      s_val[lp] = v_it[it];
    }
  }
  __syncthreads();
  const int64_t tbase = b * kOsTile;
  const int n_tile = (int)((n - tbase) < kOsTile ? (n - tbase) : kOsTile);
  for (int lp = tid; lp < n_tile; lp += kThreads) {
    const uint32_t k = s_key[lp];
    const uint32_t d = (k >> shift) & 0xffu;
    const uint32_t pos = blk_off[d] + ((uint32_t)lp - t_start[d]);
    kout[pos] = k;
    vout[pos] = s_val[lp];
  }
}



// One pass, ranked block-wide (for inputs of many waves of tiles): the
// tile's digit counts come from a shared histogram, the look-back publishes
// the tile's inclusive prefix before the ranking; then the keys are ranked
// item by item (a round of 256 keys in (item, thread) order per step, warp
// matches for equal digits, warps in order) and scattered.
__global__ void __launch_bounds__(kThreads, 4) k_os_pass_block(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
    const uint32_t* __restrict__ ghist, uint64_t* status, uint32_t* ticket, uint32_t epoch,
    unsigned* err) {
  __shared__ uint32_t s_b;
  __shared__ uint32_t blk_off[kRadix];
  __shared__ uint32_t cnt[kRadix];
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t run[kRadix];
  __shared__ uint32_t warp_sums[kWarps];
  __shared__ uint32_t t_start[kRadix];      // the tile's keys before digit d
  __shared__ uint32_t s_key[kOsTile];       // the tile in sorted order
  __shared__ uint32_t s_val[kOsTile];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_b = atomicAdd(ticket, 1u);
  cnt[tid] = 0;
  run[tid] = 0;
  __syncthreads();
  const int64_t b = s_b;
  const int64_t base = b * kOsTile;
  // this tile's digit counts
  uint32_t k_it[kOsItems], v_it[kOsItems];
#pragma unroll
  for (int it = 0; it < kOsItems; ++it) {
    const int64_t i = base + (int64_t)it * kThreads + tid;
    k_it[it] = 0;
    v_it[it] = 0;
    if (i < n) {
      k_it[it] = kin[i];
      v_it[it] = vin[i];
      atomicAdd(&cnt[(k_it[it] >> shift) & 0xffu], 1u);
    }
  }
  __syncthreads();
  // global exclusive offset of digit tid, and the tile's own
  uint32_t tot;
  const uint32_t g_excl = block_exclusive_scan(ghist[tid], warp_sums, tot);
  const uint32_t c = cnt[tid];
  t_start[tid] = block_exclusive_scan(c, warp_sums, tot);
  // publish the count, look back for the prefix, publish the prefix
  volatile uint64_t* st = status;
  if (b == 0) {
    st[(size_t)tid] = os_word(epoch, kInc, c);
    blk_off[tid] = g_excl;
  } else {
    st[(size_t)b * kRadix + tid] = os_word(epoch, kAgg, c);
    // look back 8 predecessors per step (independent loads), summing in order
    // until an inclusive prefix; a predecessor not yet published is re-read
    uint32_t prefix = 0;
    int64_t j = b - 1;
    uint32_t spins = 0;
    const long long t0 = clock64();
    bool done = false;
    while (j >= 0 && !done) {
      uint64_t wv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) wv[q] = (j - q >= 0) ? st[(size_t)(j - q) * kRadix + tid] : 0;
      int q = 0;
      for (; q < 8 && j - q >= 0; ++q) {
        const uint64_t w = wv[q];
        const uint64_t kind = (w >> 32) & 3u;
        if ((uint32_t)(w >> 34) != epoch || kind == 0) break;   // not ready yet
        prefix += (uint32_t)w;
        if (kind == kInc) {
          done = true;
          break;
        }
      }
      if (done) break;
      j -= q;
      if (q < 8 && j >= 0) {
        // never expected to take long: give up after ~1 s and record it
        if ((++spins & 63u) == 0 && clock64() - t0 > 2000000000LL) {
          set_error(err, ERR_TIMEOUT);
          break;
        }
      }
    }
    st[(size_t)b * kRadix + tid] = os_word(epoch, kInc, prefix + c);
    blk_off[tid] = g_excl + prefix;
  }
  __syncthreads();
  // stable ranks in (item, thread) order: the tile sorted in shared memory,
  // then written out in runs per digit (consecutive threads, consecutive
  // positions), instead of one scattered 4-byte store per key
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < kOsItems; ++it) {
    const int64_t i = base + (int64_t)it * kThreads + tid;
    const bool valid = i < n;
    const unsigned d = valid ? ((k_it[it] >> shift) & 0xffu) : (unsigned)kRadix;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2) wcnt[w2][tid] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t r = run[tid];
#pragma unroll
      for (int w2 = 0; w2 < kWarps; ++w2) {
        const uint32_t cc = wcnt[w2][tid];
        wcnt[w2][tid] = r;
        r += cc;
      }
      run[tid] = r;
    }
    __syncthreads();
    if (valid) {
      const uint32_t lp = t_start[d] + wcnt[wid][d] + rank;
      s_key[lp] = k_it[it];
      s_val[lp] = v_it[it];
    }
    __syncthreads();   // wcnt is cleared for the next item
  }
  const int n_tile = (int)((n - base) < kOsTile ? (n - base) : kOsTile);
  for (int lp = tid; lp < n_tile; lp += kThreads) {
    const uint32_t k = s_key[lp];
    const uint32_t d = (k >> shift) & 0xffu;
    const uint32_t pos = blk_off[d] + ((uint32_t)lp - t_start[d]);
    kout[pos] = k;
    vout[pos] = s_val[lp];
  }
}

}  // namespace

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                           SortWork& w, cudaStream_t s, uint32_t** out_keys,
                           uint32_t** out_vals) {
  *out_keys = keys;
  *out_vals = vals;
  if (n <= 0) return cudaSuccess;
  const int npass = (key_bits + 7) / 8;
  const int nblk = (int)ceil_div(n, kOsTile);
  cudaError_t e = ensure_work<uint32_t>(w, n, (int)ceil_div(n, kTileKeys), s);
  if (e != cudaSuccess) return e;
  if (w.cap_status < (size_t)nblk * kRadix) {
    dfree(w.status, s);
    w.cap_status = 0;
    if ((e = dalloc(&w.status, (size_t)nblk * kRadix, s)) != cudaSuccess) return e;
    // a fresh array holds no word of a live epoch
    if ((e = cudaMemsetAsync(w.status, 0, sizeof(uint64_t) * (size_t)nblk * kRadix, s)) !=
        cudaSuccess)
      return e;
    w.cap_status = (size_t)nblk * kRadix;
  }
  if (!w.os_meta) {
    if ((e = dalloc(&w.os_meta, (size_t)(kMaxPasses * kRadix + kMaxPasses), s)) != cudaSuccess)
      return e;
  }
  uint32_t* ghist = w.os_meta;
  uint32_t* tickets = w.os_meta + kMaxPasses * kRadix;
  e = cudaMemsetAsync(w.os_meta, 0, sizeof(uint32_t) * (kMaxPasses * kRadix + kMaxPasses), s);
  if (e != cudaSuccess) return e;
  const int hblk = (int)std::min<int64_t>(ceil_div(n, kThreads * 8), 1024);
  k_os_hist<<<hblk, kThreads, 0, s>>>(keys, n, npass, ghist);
  uint32_t *kin = keys, *kout = static_cast<uint32_t*>(w.keys_alt);
  uint32_t *vin = vals, *vout = w.vals_alt;
  // Warp-ranked passes are faster while the tiles run as one wave (their
  // look-back waits overlap the ranking); with many waves of tiles the
  // block-ranked pass keeps more tiles in flight (measured on GB300: 1e6
  // keys 0.081 vs 0.098 ms, 1e8 keys 8.4 vs 7.6 ms for the sort).
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool warp_ranked = nblk <= 2 * nsm;
  for (int p = 0; p < npass; ++p) {
    w.epoch = (w.epoch + 1) & 0x3fffffffu;
    if (w.epoch == 0) w.epoch = 1;
    if (warp_ranked)
      k_os_pass_warp<<<nblk, kThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * p,
                                               ghist + p * kRadix, w.status, tickets + p,
                                               w.epoch, w.err);
    else
      k_os_pass_block<<<nblk, kThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * p,
                                                ghist + p * kRadix, w.status, tickets + p,
                                                w.epoch, w.err);
    uint32_t* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
  *out_keys = kin;
  *out_vals = vin;
  return cudaGetLastError();
}

// Same passes as radix_sort_u32 on caller-provided scratch (no allocation):
// keys_alt / vals_alt hold n entries, hist 256 * ceil(n / 4096), totals 256.
cudaError_t radix_sort_u32_scratch(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                   uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist,
                                   uint32_t* totals, cudaStream_t s, uint32_t** out_keys,
                                   uint32_t** out_vals) {
  *out_keys = keys;
  *out_vals = vals;
  if (n <= 0) return cudaSuccess;
  const int nblk = (int)ceil_div(n, kTileKeys);
  uint32_t *kin = keys, *kout = keys_alt, *vin = vals, *vout = vals_alt;
  for (int shift = 0; shift < key_bits; shift += 8) {
    cudaError_t e = cudaMemsetAsync(totals, 0, kRadix * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_hist<uint32_t><<<nblk, kThreads, 0, s>>>(kin, n, shift, hist, totals, nblk);
    k_scan<<<kRadix, kThreads, 0, s>>>(hist, totals, nblk);
    k_scatter<uint32_t><<<nblk, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist, nblk);
    uint32_t* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
  *out_keys = kin;
  *out_vals = vin;
  return cudaGetLastError();
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                           SortWork& w, cudaStream_t s, uint64_t** out_keys,
                           uint32_t** out_vals) {
  return radix_sort_impl<uint64_t>(keys, vals, n, key_bits, w, s, out_keys, out_vals);
}

}  // namespace cg
