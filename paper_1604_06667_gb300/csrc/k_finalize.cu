// k_finalize.cu -- normalisation (paper Eq. 3; Sect. 2.1 algorithm step 3):
// R_pc = N_pc / W_p, NaN where W_p = 0, written in the caller's target order
// as [P][C] (pixel-major) or [C][P] (channel-major, the FITS cube order).
#include "cg_common.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

__global__ void k_finalize(const float* __restrict__ num, const float2* __restrict__ wsum,
                           const uint32_t* __restrict__ perm, int64_t slots, int C, int64_t P,
                           int channel_major, float* __restrict__ out,
                           float* __restrict__ out_w) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= slots * C) return;
  const int64_t slot = e / C;
  const int c = (int)(e - slot * C);
  const uint32_t u = perm[slot];
  if (u == 0xffffffffu) return;
  const float2 w2 = wsum[slot];
  const float W = w2.x + w2.y;
  const float r = (W > 0.f) ? num[e] / W : __int_as_float(0x7fc00000);
  if (channel_major) out[(size_t)c * P + u] = r;
  else out[(size_t)u * C + c] = r;
  if (out_w && c == 0) out_w[u] = W;
}

}  // namespace

cudaError_t finalize_maps(cg_grid* g, float* out, int channel_major, float* out_w) {
  const int64_t slots = g->n_slots;
  const int64_t total = slots * g->C;
  k_finalize<<<ceil_div(total, 256), 256, 0, g->stream>>>(g->acc_num, g->acc_w, g->tgt_perm,
                                                         slots, g->C, g->P, channel_major, out,
                                                         out_w);
  g->n_launches += 1;
  return cudaGetLastError();
}

}  // namespace cg
