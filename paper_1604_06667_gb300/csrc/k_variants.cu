// k_variants.cu -- gridding with one weight per sample and channel.
//
// Eq. 1-3 with omega_n replaced by omega_nc: N_pc = sum_n omega_nc w_pn D_nc,
// W_pc = sum_n omega_nc w_pn, R_pc = N_pc / W_pc.  Both sums are the gridding
// of a channel row, so one pass of the FP32 gridder over the 2C "channels"
// (omega_nc D_nc | omega_nc) with unit sample weights gives them together;
// the finalize divides channel c by channel C + c.
#include <cuda_bf16.h>

#include "cg_common.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

template <typename DT>
__device__ __forceinline__ float load_val(const DT* p);
template <>
__device__ __forceinline__ float load_val<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float load_val<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <typename DT>
__global__ void k_pcw_pack(const DT* __restrict__ data, const float* __restrict__ omega,
                           int64_t n, int C, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * C) return;
  const int64_t s = e / C;
  const int c = (int)(e % C);
  const float w = omega[e];
  const float v = load_val<DT>(data + e);
  out[s * 2 * C + c] = (w != 0.f) ? w * v : 0.f;   // a zero weight drops the value (even NaN)
  out[s * 2 * C + C + c] = w;
}

// One thread per (slot, channel): R = N / W (NaN where W <= 0), W.
__global__ void k_pcw_finalize(const float* __restrict__ acc, const uint32_t* __restrict__ perm,
                               int64_t n_slots, int C, int64_t P, int channel_major,
                               float* __restrict__ out, float* __restrict__ out_w) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_slots * C) return;
  const int64_t slot = e / C;
  const int c = (int)(e % C);
  const uint32_t u = perm[slot];
  if (u == 0xffffffffu) return;
  const float N = acc[slot * 2 * C + c];
  const float W = acc[slot * 2 * C + C + c];
  const float R = (W > 0.f) ? N / W : __int_as_float(0x7fc00000);
  if (channel_major) {
    out[(int64_t)c * P + u] = R;
    if (out_w) out_w[(int64_t)c * P + u] = W;
  } else {
    out[(int64_t)u * C + c] = R;
    if (out_w) out_w[(int64_t)u * C + c] = W;
  }
}

}  // namespace

cudaError_t pcw_pack(cg_grid* g, const void* data, int dtype, const float* omega, int64_t n) {
  cudaStream_t s = g->stream;
  const size_t need = (size_t)n * 2 * (size_t)g->C;
  cudaError_t e;
  if (g->pcw_cap_data < need) {
    dfree(g->pcw_data, s);
    g->pcw_cap_data = 0;
    if ((e = dalloc(&g->pcw_data, need, s)) != cudaSuccess) return e;
    g->pcw_cap_data = need;
  }
  if (!g->pcw_acc) {
    if ((e = dalloc(&g->pcw_acc, (size_t)g->n_slots * 2 * (size_t)g->C, s)) != cudaSuccess)
      return e;
    if ((e = dalloc(&g->pcw_w, (size_t)g->n_slots, s)) != cudaSuccess) return e;
  }
  const int64_t m = n * g->C;
  if (m == 0) return cudaSuccess;
  if (dtype == CG_BF16)
    k_pcw_pack<__nv_bfloat16><<<ceil_div(m, 256), 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(data), omega, n, g->C, g->pcw_data);
  else
    k_pcw_pack<float><<<ceil_div(m, 256), 256, 0, s>>>(static_cast<const float*>(data), omega, n,
                                                       g->C, g->pcw_data);
  g->n_launches += 1;
  return cudaGetLastError();
}

cudaError_t pcw_finalize(cg_grid* g, float* out, int channel_major, float* out_w) {
  const int64_t m = g->n_slots * (int64_t)g->C;
  if (m == 0) return cudaSuccess;
  k_pcw_finalize<<<ceil_div(m, 256), 256, 0, g->stream>>>(g->pcw_acc, g->tgt_perm, g->n_slots,
                                                          g->C, g->P, channel_major, out, out_w);
  g->n_launches += 1;
  return cudaGetLastError();
}

}  // namespace cg
