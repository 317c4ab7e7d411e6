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

}  // namespace

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                           SortWork& w, cudaStream_t s, uint32_t** out_keys,
                           uint32_t** out_vals) {
  return radix_sort_impl<uint32_t>(keys, vals, n, key_bits, w, s, out_keys, out_vals);
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
