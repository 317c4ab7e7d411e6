// k_noalloc.cu -- the sample index (RING keys + stable radix sort) for callers
// that cannot allocate device memory.  All scratch is one file-scope static
// device array; its device address is looked up once per device.
#include <mutex>

#include "cg_common.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

constexpr int64_t kMaxN = CG_NOALLOC_MAX_SAMPLES;
constexpr int64_t kMaxBlk = kMaxN / 1024;  // >= ceil(n / sort tile) for any n <= kMaxN

struct NoAllocScratch {
  uint32_t keys[2][kMaxN];
  uint32_t vals[2][kMaxN];
  uint32_t hist[256 * kMaxBlk];
  uint32_t totals[256];
};

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array for the current device (set-up on first use).
cudaError_t scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_keys_noalloc(int64_t ns, const double* __restrict__ lon,
                               const double* __restrict__ lat, int64_t n,
                               uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo = lon[i], la = lat[i];
  const bool ok = isfinite(lo) && isfinite(la) && la >= -90.0 && la <= 90.0;
  key[i] = ok ? (uint32_t)ang2pix_ring_f64(ns, lo, la) : (uint32_t)(12 * ns * ns);
  val[i] = (uint32_t)i;
}

__global__ void k_export_noalloc(const uint32_t* __restrict__ skey,
                                 const uint32_t* __restrict__ sval, int64_t n,
                                 int64_t* __restrict__ pix, int64_t* __restrict__ perm) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  pix[s] = skey[s];
  perm[s] = sval[s];
}

int key_bits(int64_t ns) {
  const uint64_t maxkey = (uint64_t)(12 * ns * ns);
  int b = 0;
  while (b < 32 && (maxkey >> b) != 0) ++b;
  return b;
}

}  // namespace

cudaError_t sort_samples_noalloc(int nside, const double* lon, const double* lat, int64_t n,
                                 int64_t* sorted_pix, int64_t* perm, cudaStream_t s) {
  NoAllocScratch* sc = nullptr;
  cudaError_t e = scratch_for_current_device(&sc);
  if (e != cudaSuccess || n == 0) return e;
  uint32_t* k0 = sc->keys[0];
  uint32_t* v0 = sc->vals[0];
  k_keys_noalloc<<<ceil_div(n, 256), 256, 0, s>>>(nside, lon, lat, n, k0, v0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t *sk = nullptr, *sv = nullptr;
  e = radix_sort_u32_scratch(k0, v0, n, key_bits(nside), sc->keys[1], sc->vals[1], sc->hist,
                             sc->totals, s, &sk, &sv);
  if (e != cudaSuccess) return e;
  k_export_noalloc<<<ceil_div(n, 256), 256, 0, s>>>(sk, sv, n, sorted_pix, perm);
  return cudaGetLastError();
}

}  // namespace cg
