// k_degrid.cu -- the adjoint of the normalised gridding operator and its
// derivative with respect to the kernel width.
//
// Gridding (Eq. 1-3) is linear in the data: R = G D with
// G[p][n] = omega_n w_pn / W_p.  The degridder applies the transpose,
//   xhat[n][c] = sum_p G[p][n] y[p][c],
// as a *gather* per sample, so that no two threads write the same output:
//   targets  RING key of every target at the handle's nside, a stable sort,
//            ring offsets and double-float unit vectors in sorted order (the
//            sample index of k_healpix.cu, built for the targets once per
//            cg_set_kernel);
//   samples  one warp per 32 consecutive sorted samples of the last add (a
//            compact strip of one HEALPix ring); its bounding disc, widened by
//            the support, is queried ring by ring (the per-ring intervals of
//            the paper's Sect. 3.3) against the target index, and every lane
//            sums the contributions of the candidate targets to its sample.
// The weights are those of the forward FP32 path (chord between double-float
// unit vectors, d^2 series or 2 asin(c/2), FP64 guard band on the cut).
//
// d/dsigma (circular Gaussian, support r fixed): w' = w d^2 / sigma^3, and
//   dR_pc/dsigma = (N'_pc - R_pc W'_p) / W_p
// with N', W' the sums of Eq. 1-2 taken with w' in place of w -- the FP32
// gridder run once with w and once with w' into scratch accumulators, then an
// epilogue that forms dR and, given an upstream gradient g, the scalar
// sum_pc g_pc dR_pc with a deterministic two-level FP64 reduction.
#include "cg_common.cuh"
#include "cg_cut.cuh"
#include "cg_healpix.cuh"
#include "cg_internal.h"
#include "cg_trig.cuh"

namespace cg {
namespace {

// ---- target index ----------------------------------------------------------
__global__ void k_target_keys(int64_t ns, const double2* __restrict__ tll,
                              const uint32_t* __restrict__ perm, int64_t n_slots,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                              float4* __restrict__ u_hi, float4* __restrict__ u_lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  val[i] = (uint32_t)i;
  const double2 ll = tll[i];
  if (perm[i] == 0xffffffffu || !valid_coord(ll.x, ll.y)) {
    key[i] = (uint32_t)(12 * ns * ns);
    u_hi[i] = make_float4(4.f, 4.f, 4.f, 0.f);
    u_lo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  df32 sb, cb, sl, cl;
  df_sincos_deg(ll.y, sb, cb);
  df_sincos_deg(ll.x, sl, cl);
  key[i] = (uint32_t)ang2pix_ring_dual(ns, ll.x, ll.y, sb);
  const df32 x = df_mul(cb, cl), y = df_mul(cb, sl);
  u_hi[i] = make_float4(x.hi, y.hi, sb.hi, 0.f);
  u_lo[i] = make_float4(x.lo, y.lo, sb.lo, 0.f);
}

// 1 / W per slot from a user-order weight map, or from the handle's
// double-float accumulator (slot order); 0 where W <= 0 or not finite.
// Normalised interpolation: every valid target slot gets the factor 1.
__global__ void k_interp_invw(const uint32_t* __restrict__ perm, int64_t n_slots,
                              float* __restrict__ invw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_slots) invw[i] = (perm[i] != 0xffffffffu) ? 1.f : 0.f;
}

__global__ void k_degrid_invw(const float* __restrict__ wmap, const float2* __restrict__ acc_w,
                              const uint32_t* __restrict__ perm, int64_t n_slots,
                              float* __restrict__ invw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  const uint32_t u = perm[i];
  float W = 0.f;
  if (u != 0xffffffffu) {
    if (wmap) {
      W = wmap[u];
    } else {
      const float2 a = acc_w[i];
      W = a.x + a.y;
    }
  }
  invw[i] = (W > 0.f && isfinite(W)) ? 1.f / W : 0.f;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct DegridArgs {
  int64_t ns;
  // samples of the last add, sorted
  const uint32_t* skey;
  const uint32_t* sval;
  const float4* s_hi;
  const float4* s_lo;
  const double2* sll;       // input order FP64 lon/lat
  int64_t n;
  // target index
  const uint32_t* t_key;    // sorted
  const uint32_t* t_slot;
  const float4* t_hi;
  const float4* t_lo;
  const int32_t* t_ring_off;
  // per slot
  const float4* f1;
  const float4* f2;
  const double2* tll;
  const uint32_t* perm;
  const float* invw;
  // operator
  KernelDev kd;
  // map and output
  const float* y;           // [P][C]
  float* out;               // [N][C]
  int C;
  unsigned* err;
  // normalised interpolation: coefficients w_pn (no sample weight, invw = 1),
  // out = sum w y / sum w (NaN where no target is within r), vsum = sum w
  int interp;
  float* vsum;              // [N] or null
};

// One warp per 32 consecutive sorted samples; CB channels per pass (grid.y
// covers the channel blocks).
template <int CB, int KT, bool BIG>
__global__ void __launch_bounds__(256) k_degrid(DegridArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t wt = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int64_t s = wt * 32 + lane;
  if (wt * 32 >= a.n) return;
  const int c_base = blockIdx.y * CB;
  const int64_t npix = 12 * a.ns * a.ns;
  const bool in_range = s < a.n;
  const bool live = in_range && (int64_t)a.skey[s] < npix;
  float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
  uint32_t idx = 0;
  double2 sll = make_double2(0.0, 0.0);
  if (in_range) idx = a.sval[s];
  if (live) {
    h = a.s_hi[s];
    l = a.s_lo[s];
    sll = a.sll[idx];
  }
  float x[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = 0.f;
  float vs = 0.f;   // sum of this sample's coefficients (interpolation)

  // ---- segments: runs of live samples whose neighbours (in sorted order)
  // lie within the support radius; a run that crosses into the next ring or
  // over a gap in the coverage starts a new segment with its own query ----
  const float seg_c = 2.f * sinf(0.5f * (float)a.kd.r_rad);
  const float px = __shfl_up_sync(0xffffffffu, h.x, 1);
  const float py = __shfl_up_sync(0xffffffffu, h.y, 1);
  const float pz = __shfl_up_sync(0xffffffffu, h.z, 1);
  const bool plive = __shfl_up_sync(0xffffffffu, live, 1);
  bool start = false;
  if (live) {
    const float gx = h.x - px, gy = h.y - py, gz = h.z - pz;
    start = lane == 0 || !plive || (gx * gx + gy * gy + gz * gz) > seg_c * seg_c;
  }
  const uint32_t starts = __ballot_sync(0xffffffffu, start);
  const int seg_id = __popc(starts & ((2u << lane) - 1u)) - 1;   // -1 before the first
  const int n_seg = __popc(starts);
  for (int seg = 0; seg < n_seg; ++seg) {
    const bool mine = live && seg_id == seg;
    // bounding disc of the segment
    float sx = mine ? h.x : 0.f, sy = mine ? h.y : 0.f, sz = mine ? h.z : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    const float nrm = sqrtf(sx * sx + sy * sy + sz * sz);
    if (!(nrm > 0.f)) continue;
    const float cx = sx / nrm, cy = sy / nrm, cz = sz / nrm;
    float ch = 0.f;
    if (mine) {
      const float ex = h.x - cx, ey = h.y - cy, ez = h.z - cz;
      ch = sqrtf(ex * ex + ey * ey + ez * ez);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ch = fmaxf(ch, __shfl_xor_sync(0xffffffffu, ch, o));
    const double rt = 2.0 * asin(fmin(1.0, 0.5 * (double)ch)) * (1.0 + 1e-5) + 1e-6;
    Disc disc;
    disc.tc = acos(fmin(1.0, fmax(-1.0, (double)cz)));
    disc.pc = atan2((double)cy, (double)cx);
    disc.R = rt + a.kd.r_rad + 1e-6;
    const double tlo = fmax(0.0, disc.tc - disc.R), thi = fmin(kPi, disc.tc + disc.R);
    int64_t ilo = (int64_t)floor(ring_coord(a.ns, cos(tlo))) - 2;
    int64_t ihi = (int64_t)ceil(ring_coord(a.ns, cos(thi))) + 2;
    ilo = ilo < 1 ? 1 : ilo;
    ihi = ihi > 4 * a.ns - 1 ? 4 * a.ns - 1 : ihi;
    const float q1 = a.kd.k1, q2 = a.kd.k2;
    for (int64_t base = ilo; base <= ihi; base += 32) {
      // lane j: the target interval(s) of ring base + j
      const int64_t ring = base + lane;
      int2 iv[2] = {make_int2(0, 0), make_int2(0, 0)};
      if (ring <= ihi) {
        Range rr[2];
        const int nr = ring_ranges(a.ns, ring, &disc, 1, rr);
        const int32_t ta = a.t_ring_off[ring], tb = a.t_ring_off[ring + 1];
        for (int q = 0; q < nr && tb > ta; ++q) {
          const int32_t lo = lower_bound_u32(a.t_key, ta, tb, (uint32_t)rr[q].pix_lo);
          const int32_t hi = lower_bound_u32(a.t_key, lo, tb, (uint32_t)rr[q].pix_hi + 1u);
          iv[q] = make_int2(lo, hi);
        }
      }
      for (int j = 0; j < 32; ++j) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t0 = __shfl_sync(0xffffffffu, iv[q].x, j);
          const int t1 = __shfl_sync(0xffffffffu, iv[q].y, j);
          for (int t = t0; t < t1; ++t) {
            const uint32_t slot = a.t_slot[t];
            const float iw = a.invw[slot];
            if (iw == 0.f) continue;        // W_p = 0: the row of G is zero
            const float4 th = a.t_hi[t], tl = a.t_lo[t];
            const float dx = df_diff(h.x, l.x, th.x, tl.x);
            const float dy = df_diff(h.y, l.y, th.y, tl.y);
            const float dz = df_diff(h.z, l.z, th.z, tl.z);
            const float c2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float coef = 0.f;
            if (mine && c2 <= a.kd.c2_out) {
              float d2;
              if (!BIG) {
                d2 = c2 * fmaf(c2, fmaf(c2, 1.f / 90.f, 1.f / 12.f), 1.f);
              } else {
                const float d = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(c2)));
                d2 = d * d;
              }
              float ex;
              if (KT == CG_GAUSS1D || KT == CG_TSINC) {
                ex = q1 * d2;
              } else {
                const float4 f1 = a.f1[slot], f2 = a.f2[slot];
                const float ap = fmaf(dx, f1.x, fmaf(dy, f1.y, dz * f1.z));
                const float bp = fmaf(dx, f2.x, fmaf(dy, f2.y, dz * f2.z));
                const float s2 = fmaf(ap, ap, bp * bp);
                const float ratio = (s2 > 0.f) ? __fdividef(d2, s2) : 1.f;
                ex = fmaf(q1 * ap, ap, q2 * bp * bp) * ratio;
              }
              coef = ex2_approx(ex) * (a.interp ? 1.f : h.w) * iw;
              if (KT == CG_TSINC) coef *= sinc_pi(sqrtf(d2) * a.kd.inv_a);
              if (c2 >= a.kd.c2_in) {
                if (!pair_inside(a.tll[slot], sll, a.kd.c2r_hi, a.kd.c2r_lo, a.kd.c2r_tol,
                                 a.kd.r_rad))
                  coef = 0.f;
              }
            }
            vs += coef;
            if (!__any_sync(0xffffffffu, coef != 0.f)) continue;
            const float* yr = a.y + (size_t)a.perm[slot] * a.C + c_base;
#pragma unroll
            for (int c = 0; c < CB; ++c)
              if (c_base + c < a.C) x[c] = fmaf(coef, __ldg(yr + c), x[c]);
          }
        }
      }
    }
  }
  if (in_range) {
    float* o = a.out + (size_t)idx * a.C + c_base;
    if (a.interp) {
      const float inv = (vs > 0.f) ? 1.f / vs : __int_as_float(0x7fc00000);
#pragma unroll
      for (int c = 0; c < CB; ++c) x[c] *= inv;
      if (a.vsum && blockIdx.y == 0) a.vsum[idx] = vs;
    }
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (c_base + c < a.C) o[c] = x[c];
  }
}

template <int CB>
cudaError_t launch_degrid(const DegridArgs& a, bool big, cudaStream_t s) {
  const int64_t warps = (a.n + 31) / 32;
  const dim3 grid((unsigned)((warps + 7) / 8), (unsigned)((a.C + CB - 1) / CB));
  if (a.kd.type == CG_GAUSS1D) {
    if (big) k_degrid<CB, CG_GAUSS1D, true><<<grid, 256, 0, s>>>(a);
    else k_degrid<CB, CG_GAUSS1D, false><<<grid, 256, 0, s>>>(a);
  } else if (a.kd.type == CG_TSINC) {
    k_degrid<CB, CG_TSINC, true><<<grid, 256, 0, s>>>(a);
  } else {
    if (big) k_degrid<CB, CG_GAUSS2D, true><<<grid, 256, 0, s>>>(a);
    else k_degrid<CB, CG_GAUSS2D, false><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---- d/dsigma epilogue -----------------------------------------------------
constexpr int kDsBlock = 256;

// dR[user][c] = (N' - R W') / W (NaN where W = 0) and the block's share of
// sum g dR (FP64) -- one thread per (slot, channel).
__global__ void __launch_bounds__(kDsBlock) k_dsigma_out(
    const float* __restrict__ n0, const float2* __restrict__ w0, const float* __restrict__ n1,
    const float2* __restrict__ w1, const uint32_t* __restrict__ perm, int64_t n_slots, int C,
    const float* __restrict__ grad, float* __restrict__ dR, double* __restrict__ part) {
  __shared__ double red[kDsBlock / 32];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (e < n_slots * C) {
    const int64_t slot = e / C;
    const int c = (int)(e % C);
    const uint32_t u = perm[slot];
    if (u != 0xffffffffu) {
      const float2 a0 = w0[slot], a1 = w1[slot];
      const double W = (double)a0.x + (double)a0.y;
      const double Wp = (double)a1.x + (double)a1.y;
      double v = __int_as_float(0x7fc00000);
      if (W > 0.0) {
        const double R = (double)n0[slot * C + c] / W;
        v = ((double)n1[slot * C + c] - R * Wp) / W;
        if (grad) acc = (double)grad[(size_t)u * C + c] * v;
      }
      if (dR) dR[(size_t)u * C + c] = (float)v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kDsBlock / 32; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

// One block: fixed-order sum of the block partials.
__global__ void __launch_bounds__(kDsBlock) k_dsigma_sum(const double* __restrict__ part,
                                                         int64_t nb, double* __restrict__ out) {
  __shared__ double red[kDsBlock];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < nb; i += kDsBlock) t += part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = kDsBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

// Build (once per cg_set_kernel) the sorted RING index of the targets.
cudaError_t target_index_build(cg_grid* g) {
  if (g->tix_valid) return cudaSuccess;
  cudaStream_t s = g->stream;
  const int64_t m = g->n_slots;
  cudaError_t e;
  dfree(g->tix_ring_off, s);
  if (!g->tix_key) {
    if ((e = dalloc(&g->tix_key, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_val, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_uhi, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_ulo, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_hi, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_lo, (size_t)m, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->tix_invw, (size_t)m, s)) != cudaSuccess) return e;
  }
  if ((e = dalloc(&g->tix_ring_off, (size_t)(4 * g->nside + 1), s)) != cudaSuccess) return e;
  k_target_keys<<<ceil_div(m, 256), 256, 0, s>>>(g->nside, g->tgt_ll, g->tgt_perm, m, g->tix_key,
                                                 g->tix_val, g->tix_uhi, g->tix_ulo);
  g->n_launches += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int bits = key_bits_for(g->nside);
  g->tix_sw.err = g->d_err;
  if ((e = radix_sort_u32(g->tix_key, g->tix_val, m, bits, g->tix_sw, s, &g->tix_skey,
                          &g->tix_sslot)) != cudaSuccess)
    return e;
  g->n_launches += 1 + (bits + 7) / 8;
  if ((e = sorted_gather(g->nside, g->tix_skey, g->tix_sslot, g->tix_uhi, g->tix_ulo, 1, m,
                         g->tix_hi, g->tix_lo, g->tix_ring_off, s)) != cudaSuccess)
    return e;
  g->n_launches += 1;
  g->tix_valid = true;
  return cudaSuccess;
}

cudaError_t grid_degrid(cg_grid* g, const float* y, const float* wmap, float* out, bool interp,
                        float* vsum) {
  cudaStream_t s = g->stream;
  cudaError_t e = target_index_build(g);
  if (e != cudaSuccess) return e;
  if (interp)
    k_interp_invw<<<ceil_div(g->n_slots, 256), 256, 0, s>>>(g->tgt_perm, g->n_slots, g->tix_invw);
  else
    k_degrid_invw<<<ceil_div(g->n_slots, 256), 256, 0, s>>>(wmap, g->acc_w, g->tgt_perm,
                                                            g->n_slots, g->tix_invw);
  g->n_launches += 1;
  DegridArgs a;
  a.ns = g->nside;
  a.skey = g->sorted_key;
  a.sval = g->sorted_val;
  a.s_hi = g->s_hi;
  a.s_lo = g->s_lo;
  a.sll = g->s_ll;
  a.n = g->last_n;
  a.t_key = g->tix_skey;
  a.t_slot = g->tix_sslot;
  a.t_hi = g->tix_hi;
  a.t_lo = g->tix_lo;
  a.t_ring_off = g->tix_ring_off;
  a.f1 = g->tgt_f1;
  a.f2 = g->tgt_f2;
  a.tll = g->tgt_ll;
  a.perm = g->tgt_perm;
  a.invw = g->tix_invw;
  a.kd = g->kdev;
  a.y = y;
  a.out = out;
  a.C = g->C;
  a.err = g->d_err;
  a.interp = interp ? 1 : 0;
  a.vsum = vsum;
  if (a.n == 0) return cudaGetLastError();
  g->n_launches += 1;
  const bool big = g->kdev.big_support != 0;
  if (g->C <= 8) return launch_degrid<8>(a, big, s);
  if (g->C <= 16) return launch_degrid<16>(a, big, s);
  return launch_degrid<32>(a, big, s);
}

cudaError_t grid_dsigma(cg_grid* g, const void* data, int dtype, const float* grad, float* dR,
                        double* dsigma) {
  cudaStream_t s = g->stream;
  const size_t ns = (size_t)g->n_slots, C = (size_t)g->C;
  cudaError_t e;
  if (!g->ds_num) {
    if ((e = dalloc(&g->ds_num, ns * C, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->ds_w, ns, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->ds_num0, ns * C, s)) != cudaSuccess) return e;
    if ((e = dalloc(&g->ds_w0, ns, s)) != cudaSuccess) return e;
  }
  const int64_t total = g->n_slots * (int64_t)g->C;
  const int64_t nb = ceil_div(total, kDsBlock);
  dfree(g->ds_part, s);
  if ((e = dalloc(&g->ds_part, (size_t)(nb > 0 ? nb : 1), s)) != cudaSuccess) return e;
  // the FP32 gridder over the 64-target tiles: the per-add ranges of that
  // tiling must belong to the current sample index
  if (g->t64.ranges_gen != g->index_gen) {
    if ((e = tiles_ranges(g, g->t64)) != cudaSuccess) return e;
    g->t64.ranges_gen = g->index_gen;
  }
  // d R / d sigma with sigma in degrees: w' = w d^2 / sigma^3 with d in degrees
  const double sig = g->kparams[0];
  const double rad2deg = 180.0 / kPi;
  const float dscale = (float)(rad2deg * rad2deg / (sig * sig * sig));
  if ((e = grid_tiles_f32_to(g, data, dtype, g->ds_num0, g->ds_w0, 0, 0.f)) != cudaSuccess)
    return e;
  if ((e = grid_tiles_f32_to(g, data, dtype, g->ds_num, g->ds_w, 0, dscale)) != cudaSuccess)
    return e;
  if (nb > 0) {
    k_dsigma_out<<<(unsigned)nb, kDsBlock, 0, s>>>(g->ds_num0, g->ds_w0, g->ds_num, g->ds_w,
                                                   g->tgt_perm, g->n_slots, g->C, grad, dR,
                                                   g->ds_part);
    g->n_launches += 1;
  }
  if (dsigma) {
    k_dsigma_sum<<<1, kDsBlock, 0, s>>>(g->ds_part, nb, dsigma);
    g->n_launches += 1;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Map making by gradient descent on 1/2 ||G^T m - D||^2 (G the normalised
// gridding operator of Eq. 3, G^T its adjoint): the element-wise steps of
// one iteration, in the library.
// ---------------------------------------------------------------------------
namespace {

constexpr int kMdBlock = 256;
constexpr int kMdPer = 4;   // values per thread

// r <- r - D; per-block FP64 partial sums of r^2 (fixed order).
__global__ void __launch_bounds__(kMdBlock) k_md_residual(float* __restrict__ r,
                                                          const float* __restrict__ d, int64_t n,
                                                          double* __restrict__ part) {
  __shared__ double red[kMdBlock];
  const int64_t base = (int64_t)blockIdx.x * kMdBlock * kMdPer;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kMdPer; ++k) {
    const int64_t i = base + (int64_t)k * kMdBlock + threadIdx.x;
    if (i < n) {
      const float v = r[i] - d[i];
      r[i] = v;
      acc += (double)v * (double)v;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kMdBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss = 1/2 sum of the partials (one block, fixed order).
__global__ void __launch_bounds__(kMdBlock) k_md_loss(const double* __restrict__ part, int64_t nb,
                                                      double* __restrict__ loss) {
  __shared__ double red[kMdBlock];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < nb; i += kMdBlock) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kMdBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5 * red[0];
}

// m <- m - alpha g, where g is NaN (a target no sample reaches) taking 0.
__global__ void k_md_update(float* __restrict__ m, const float* __restrict__ g, float alpha,
                            int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = g[i];
  if (!isnan(v)) m[i] = fmaf(-alpha, v, m[i]);
}

}  // namespace

cudaError_t md_residual(cg_grid* g, float* r, const float* d, int64_t n, double* loss) {
  cudaStream_t s = g->stream;
  const int64_t nb = (n + kMdBlock * kMdPer - 1) / (kMdBlock * kMdPer);
  if ((size_t)nb > g->md_cap) {
    dfree(g->md_part, s);
    g->md_cap = 0;
    cudaError_t e = dalloc(&g->md_part, (size_t)(nb > 0 ? nb : 1), s);
    if (e != cudaSuccess) return e;
    g->md_cap = (size_t)nb;
  }
  if (nb > 0) k_md_residual<<<(unsigned)nb, kMdBlock, 0, s>>>(r, d, n, g->md_part);
  k_md_loss<<<1, kMdBlock, 0, s>>>(g->md_part, nb, loss);
  g->n_launches += nb > 0 ? 2 : 1;
  return cudaGetLastError();
}

cudaError_t md_update(cg_grid* g, float* m, const float* grad, float alpha, int64_t n) {
  if (n <= 0) return cudaSuccess;
  k_md_update<<<ceil_div(n, 256), 256, 0, g->stream>>>(m, grad, alpha, n);
  g->n_launches += 1;
  return cudaGetLastError();
}

}  // namespace cg
