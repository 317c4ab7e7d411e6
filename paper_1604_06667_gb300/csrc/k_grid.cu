// k_grid.cu -- tile gridder, FP32 CUDA-core form (paper Eq. 1-2).
//
// One CTA owns one tile of kTile targets, so no two CTAs ever write the same
// output cell: the race-free ownership of target pixels of the paper's lookup
// scheme (Sect. 2.2, "the program writes into different map and weight-map
// cells in each thread"), with a CTA in place of a CPU thread.
//
// The CTA walks the tile's candidate samples -- the sample ranges that the
// tile's disc query selected -- in chunks of kChunk, two stages deep:
//   stage    candidate unit vectors (double-float) and sample weight, and the
//            candidates' channel rows (FP32 rows by cp.async, 16-byte pieces
//            straight into shared memory, issued one chunk ahead);
//   phase A  weights w[k][p] for every (candidate, target) pair: chord between
//            tile-relative FP32 vectors, exact cut d <= r (FP64 recomputation
//            inside a narrow guard band around r), Gaussian via ex2;
//            per-target weight sums W_p with Neumaier compensation;
//   phase B  register-blocked accumulation acc[p][c] += w[k][p] * D[k][c]
//            (packed f32x2 FMAs on channel pairs),
//            skipping candidates whose weights for the thread's targets are 0.
// The epilogue adds acc into the numerator and W into the weight map (tile
// order; cg_grid_finalize applies Eq. 3 and the user layout).  A target row
// whose numerator came out non-finite (a NaN or Inf channel value reaches the
// thread's other targets through 0 x NaN) is left to k_nonfinite_fixup.
#include <cuda_bf16.h>

#include <algorithm>

#include "cg_common.cuh"
#include "cg_cut.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

constexpr int kRangeBatch = 256;


__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename DT>
__device__ __forceinline__ float load_elem(const DT* p);
template <>
__device__ __forceinline__ float load_elem<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_elem<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <typename DT>
__device__ __forceinline__ float4 load_vec4(const DT* p);
template <>
__device__ __forceinline__ float4 load_vec4<float>(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 load_vec4<__nv_bfloat16>(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  float4 r;
  r.x = __uint_as_float(u.x << 16);
  r.y = __uint_as_float(u.x & 0xffff0000u);
  r.z = __uint_as_float(u.y << 16);
  r.w = __uint_as_float(u.y & 0xffff0000u);
  return r;
}

// Weight omega w(p, k) of target p (tile-relative vector at, elliptical axes
// f1, f2) against candidate sh (tile-relative vector, omega in .w) in FP32:
// chord, exact cut d <= r (FP64 recomputation inside the guard band),
// kernel value.  Pairs outside the support get -0.0: it adds nothing to any
// finite sum, and its sign bit tells the accumulation that the pair does not
// take part at all (so that a non-finite channel value of a sample reaches
// only the targets within its support, paper Eq. 1-2).
__device__ __forceinline__ float pair_weight(const KernelDev& kd, float4 at, float4 f1, float4 f2,
                                             float4 sh, double2 tll, const double2* sll,
                                             uint32_t idx, bool& in) {
  const float dx = at.x - sh.x, dy = at.y - sh.y, dz = at.z - sh.z;
  const float c2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  in = false;
  if (!(c2 <= kd.c2_out)) return -0.f;
  float d2;
  if (!kd.big_support) {
    d2 = c2 * fmaf(c2, fmaf(c2, 1.f / 90.f, 1.f / 12.f), 1.f);
  } else {
    const float d = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(c2)));
    d2 = d * d;
  }
  float ex;
  if (kd.type == CG_GAUSS1D || kd.type == CG_TSINC) {
    ex = kd.k1 * d2;
  } else {
    const float ap = fmaf(dx, f1.x, fmaf(dy, f1.y, dz * f1.z));
    const float bp = fmaf(dx, f2.x, fmaf(dy, f2.y, dz * f2.z));
    const float s2 = fmaf(ap, ap, bp * bp);  // sin^2 d
    const float ratio = (s2 > 0.f) ? __fdividef(d2, s2) : 1.f;
    ex = fmaf(kd.k1 * ap, ap, kd.k2 * bp * bp) * ratio;
  }
  float w = ex2_approx(ex) * sh.w;
  if (kd.type == CG_TSINC) w *= sinc_pi(sqrtf(d2) * kd.inv_a);
  if (kd.dscale != 0.f) w *= d2 * kd.dscale;   // dw/dsigma pass
  in = true;
  if (c2 >= kd.c2_in) {
    // guard band: decide d <= r again from the input coordinates
    in = pair_inside_inl(tll, sll[idx], kd.c2r_hi, kd.c2r_lo, kd.c2r_tol, kd.r_rad);
  }
  return in ? w : -0.f;
}

__device__ __forceinline__ bool takes_part(float w) { return __float_as_uint(w) != 0x80000000u; }

// Shared memory of one k_grid_f32 CTA: two stages of candidates (tile-relative
// vector, input index), their channel rows (FP32) and their weights, so that
// the copies of chunk q + 1 run under the weights and the accumulation of
// chunk q.
template <int PB, int CB, int NCG>
struct alignas(16) F32Smem {
  static constexpr int NTH = (kTile / PB) * NCG;
  static constexpr int CPAD = CB * NCG;
  float d[2][kChunk][CPAD];      // channel rows of the candidates
  float w[2][kChunk][kTile];     // weights w[k][p]
  float4 b[2][kChunk];           // tile-relative candidate vectors and omega (narrow shapes: pair-major, negated)
  uint32_t idx[2][kChunk];       // input index (0xffffffff: padding)
  int2 rg[kRangeBatch];          // a batch of the tile's sample ranges
  int rg_pre[kRangeBatch + 1];   // candidates before each range of the batch
  float2 wred[NTH];
  float wfin[kTile];             // W of the tile's targets (one-shot output)
  int row_nf[kTile];             // rows of this CTA with a non-finite numerator
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous global -> shared copy; src_bytes 0 fills zeros.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
// 4-byte asynchronous global -> shared copy (scalar rows); src_bytes 0 fills zeros.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One (tile, channel slab, candidate split) item of the FP32 gridder, by a
// CTA of (kTile / PB) * NCG threads: PB targets x CB channels per thread in
// phase B, NCG channel groups.
template <int PB, int CB, int NCG, typename DT>
__device__ __forceinline__ void grid_item_f32(const GridArgs& a, F32Smem<PB, CB, NCG>& S,
                                              int64_t tile, int slab, int split, int n_slabs) {
  using Smem = F32Smem<PB, CB, NCG>;
  constexpr int NTH = Smem::NTH;
  constexpr int CPAD = Smem::CPAD;
  constexpr int K = kChunk;
  constexpr int STEP = NTH / kTile;
  static_assert(NTH % kTile == 0, "threads must cover the tile");
  static_assert(CB % 4 == 0, "channel blocks are float4 wide");

  const int tid = threadIdx.x;
  const int c_base = slab * CPAD;

  // phase-A identity: one target, every STEP-th candidate
  const int p = tid % kTile;
  const int kk0 = tid / kTile;
  const int64_t slot = tile * kTile + p;
  const float4 at = a.tgt_a[slot];
  float4 f1 = make_float4(0, 0, 0, 0), f2 = f1;
  if (a.kd.type == CG_GAUSS2D) {
    f1 = a.tgt_f1[slot];
    f2 = a.tgt_f2[slot];
  }
  const float4 chi = a.tile_chi[tile];
  const float4 clo = a.tile_clo[tile];
  float ws = 0.f, wc = 0.f;  // Neumaier sum of weights
  unsigned npair = 0;        // pairs inside the support

  // phase-B identity
  const int pg = tid / NCG;
  const int cg = tid % NCG;
  // channel sums as packed pairs (channels 2 m, 2 m + 1 of the thread's
  // blocks): one fma.rn.f32x2 does both, the same IEEE fma per lane
  float2 acc[PB][CB / 2];
#pragma unroll
  for (int i = 0; i < PB; ++i)
#pragma unroll
    for (int j = 0; j < CB / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);

  const DT* data = static_cast<const DT*>(a.data);
  const int C = a.C;
  // shapes of at most 8 channels per thread are latency-bound: they load the
  // candidate records of chunk q + 2 into registers while chunk q is
  // computed, and copy unaligned FP32 rows asynchronously element by element
  constexpr bool kPrefetch = CB <= 8;
  // narrow shapes: phase A on candidate pairs with packed f32x2 arithmetic
  // (candidate vectors stored pair-major and negated)
  constexpr bool kPairs = CB <= 8;
  // FP32 rows go straight to shared memory (cp.async: 16-byte pieces when
  // aligned); BF16 rows and the wide shapes' unaligned rows through registers
  const bool async_rows = sizeof(DT) == 4 && (a.vec4 || kPrefetch);
  const int64_t r0 = a.range_off[tile], r1 = a.range_off[tile + 1];
  // this CTA's share [c_lo, c_hi) of the tile's candidates (whole chunks)
  int c_lo = 0, c_hi = 0x7fffffff;
  if (a.n_split > 1) {
    const int total_t = a.tile_cand[tile];
    const int per = ((total_t + a.n_split - 1) / a.n_split + K - 1) / K * K;
    c_lo = split * per;
    c_hi = min(total_t, c_lo + per);
  }
  int cbase = 0;   // the tile's candidates before the current range batch

  for (int64_t rb = r0; rb < r1 && cbase < c_hi; rb += kRangeBatch) {
    const int nr = (int)((r1 - rb) < kRangeBatch ? (r1 - rb) : kRangeBatch);
    __syncthreads();   // the previous batch's chunks are done with rg / rg_pre
    if (tid < 32) {
      // warp 0: load this batch of ranges and prefix-sum their lengths
      int carry = 0;
      for (int b = 0; b < nr; b += 32) {
        const int q = b + tid;
        int len = 0;
        if (q < nr) {
          const int2 r = a.range_s[rb + q];
          S.rg[q] = r;
          len = r.y - r.x;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += y;
        }
        if (q < nr) S.rg_pre[q] = carry + incl - len;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (tid == 0) S.rg_pre[nr] = carry;
    }
    __syncthreads();
    const int total = S.rg_pre[nr];
    const int v_lo = max(0, min(total, c_lo - cbase));
    const int v_hi = max(0, min(total, c_hi - cbase));
    cbase += total;
    const int n_chunks = (v_hi - v_lo + K - 1) / K;
    if (n_chunks == 0) continue;

    // the record of candidate v0 + tid (threads tid < K): loads only
    struct Cand {
      float4 h, l;
      uint32_t idx;
    };
    auto fetch_cand = [&](int v0) {
      // padding candidate (never equal to an empty target slot's sentinel)
      Cand c{make_float4(-4.f, -4.f, -4.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), 0xffffffffu};
      const int v = v0 + tid;
      if (tid < K && v < v_hi) {
        int lo = 0, hi = nr - 1;  // last range with rg_pre <= v
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (S.rg_pre[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const int64_t s = S.rg[lo].x + (v - S.rg_pre[lo]);
        c.h = a.s_hi[s];
        c.l = a.s_lo[s];
        c.idx = a.perm[s];
      }
      return c;
    };
    // a fetched record into stage st: the candidate relative to the tile
    // centre, once for all targets
    auto put_cand = [&](const Cand& c, int st) {
      if (tid < K) {
        const float bx = df_diff(c.h.x, c.l.x, chi.x, clo.x);
        const float by = df_diff(c.h.y, c.l.y, chi.y, clo.y);
        const float bz = df_diff(c.h.z, c.l.z, chi.z, clo.z);
        if constexpr (kPairs) {
          // pair-major: (-x, -x', -y, -y'), (-z, -z', omega, omega') for the
          // candidate pair (tid & ~1, tid | 1); target + (-candidate) is the
          // target - candidate difference exactly
          float* q = reinterpret_cast<float*>(&S.b[st][tid & ~1]) + (tid & 1);
          q[0] = -bx;
          q[2] = -by;
          q[4] = -bz;
          q[6] = c.h.w;
        } else {
          S.b[st][tid] = make_float4(bx, by, bz, c.h.w);
        }
        S.idx[st][tid] = c.idx;
      }
    };
    auto stage_cands = [&](int v0, int st) { put_cand(fetch_cand(v0), st); };
    // channel rows of stage st's candidates (their indices are visible)
    auto stage_rows = [&](int st) {
      if (async_rows && a.vec4) {
        for (int e = tid; e < K * (CPAD / 4); e += NTH) {
          const int k = e / (CPAD / 4);
          const int c = (e % (CPAD / 4)) * 4;
          const uint32_t idx = S.idx[st][k];
          const bool ok = idx != 0xffffffffu && c_base + c < C;
          const DT* src = ok ? data + (size_t)idx * C + c_base + c : data;
          cp_async16(&S.d[st][k][c], src, ok ? 16 : 0);
        }
        cp_async_commit();
      } else if (a.vec4) {
        for (int e = tid; e < K * (CPAD / 4); e += NTH) {
          const int k = e / (CPAD / 4);
          const int c = (e % (CPAD / 4)) * 4;
          const uint32_t idx = S.idx[st][k];
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (idx != 0xffffffffu && c_base + c < C)
            v = load_vec4<DT>(data + (size_t)idx * C + c_base + c);
          *reinterpret_cast<float4*>(&S.d[st][k][c]) = v;
        }
      } else {
        for (int e = tid; e < K * CPAD; e += NTH) {
          const int k = e / CPAD;
          const int c = e % CPAD;
          const uint32_t idx = S.idx[st][k];
          float v = 0.f;
          if (idx != 0xffffffffu && c_base + c < C) v = load_elem<DT>(data + (size_t)idx * C + c_base + c);
          S.d[st][k][c] = v;
        }
      }
    };
    // FP32 rows of any alignment, asynchronously (4-byte elements when the
    // rows are not 16-byte aligned)
    auto stage_rows_async = [&](int st) {
      if constexpr (kPrefetch) {
        if (!a.vec4) {
          for (int e = tid; e < K * CPAD; e += NTH) {
            const int k = e / CPAD;
            const int c = e % CPAD;
            const uint32_t idx = S.idx[st][k];
            const bool ok = idx != 0xffffffffu && c_base + c < C;
            const DT* src = ok ? data + (size_t)idx * C + c_base + c : data;
            cp_async4(&S.d[st][k][c], src, ok ? 4 : 0);
          }
          cp_async_commit();
          return;
        }
      }
      stage_rows(st);
    };

    // Two-stage pipeline, one barrier per chunk.  Chunk q uses stage q & 1.
    // Before the barrier of chunk q: the candidates of chunk q + 1 and the
    // weights of chunk q; after it: the rows of chunk q + 1 are issued and
    // chunk q is accumulated.  A stage is rewritten only after the barrier
    // that follows its last reader.
    stage_cands(v_lo, 0);
    __syncthreads();
    if (async_rows) stage_rows_async(0); else stage_rows(0);
    Cand pre;   // kPrefetch: the record of chunk q + 1, loaded one chunk ago
    if (kPrefetch && n_chunks > 1) pre = fetch_cand(v_lo + K);
    for (int q = 0; q < n_chunks; ++q) {
      const int cur = q & 1, nxt = cur ^ 1;
      const bool more = q + 1 < n_chunks;
      if (kPrefetch) {
        if (more) put_cand(pre, nxt);
        if (q + 2 < n_chunks) pre = fetch_cand(v_lo + (q + 2) * K);
      } else if (more) {
        stage_cands(v_lo + (q + 1) * K, nxt);
      }

      // ---- phase A: weights ----
      // the arithmetic of pair_weight, written out, for candidate k at
      // squared chord c2 (pairs outside the support get -0.0)
      const float4* bp = S.b[cur];
      // target - candidate k
      auto diff = [&](int k) {
        if constexpr (kPairs) {
          const float* q = reinterpret_cast<const float*>(&bp[k & ~1]) + (k & 1);
          return make_float3(at.x + q[0], at.y + q[2], at.z + q[4]);
        } else {
          const float4 sh = bp[k];
          return make_float3(at.x - sh.x, at.y - sh.y, at.z - sh.z);
        }
      };
      auto one = [&](int k, float c2, float om) {
        float w = -0.f;
        if (c2 <= a.kd.c2_out) {
          float d2;
          if (!a.kd.big_support) {
            d2 = c2 * fmaf(c2, fmaf(c2, 1.f / 90.f, 1.f / 12.f), 1.f);
          } else {
            const float d = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(c2)));
            d2 = d * d;
          }
          float ex;
          if (a.kd.type == CG_GAUSS1D || a.kd.type == CG_TSINC) {
            ex = a.kd.k1 * d2;
          } else {
            const float3 dv = diff(k);
            const float dx = dv.x, dy = dv.y, dz = dv.z;
            const float ap = fmaf(dx, f1.x, fmaf(dy, f1.y, dz * f1.z));
            const float bp = fmaf(dx, f2.x, fmaf(dy, f2.y, dz * f2.z));
            const float s2 = fmaf(ap, ap, bp * bp);  // sin^2 d
            const float ratio = (s2 > 0.f) ? __fdividef(d2, s2) : 1.f;
            ex = fmaf(a.kd.k1 * ap, ap, a.kd.k2 * bp * bp) * ratio;
          }
          w = ex2_approx(ex) * om;
          if (a.kd.type == CG_TSINC) w *= sinc_pi(sqrtf(d2) * a.kd.inv_a);
          if (a.kd.dscale != 0.f) w *= d2 * a.kd.dscale;   // dw/dsigma pass
          bool in = true;
          if (c2 >= a.kd.c2_in) {
            // guard band: decide d <= r again from the input coordinates
            const uint32_t idx = S.idx[cur][k];
            in = pair_inside_inl(a.tgt_ll[slot], a.sll[idx], a.kd.c2r_hi, a.kd.c2r_lo,
                                 a.kd.c2r_tol, a.kd.r_rad);
          }
          if (in) {
            ++npair;
            // Neumaier (two-sum) accumulation of the weight map; a pair
            // outside the support adds -0.0, which leaves (ws, wc) as they are
            const float t = ws + w;
            const float bp2 = t - ws;
            wc += (ws - (t - bp2)) + (w - bp2);
            ws = t;
          } else {
            w = -0.f;
          }
        }
        S.w[cur][k][p] = w;
      };
      if constexpr (kPairs) {
        // candidates in pairs (2 j, 2 j + 1): the difference vectors and the
        // squared chords on packed f32x2 lanes, the same IEEE operations per lane
        const float2 at_x2 = make_float2(at.x, at.x), at_y2 = make_float2(at.y, at.y),
                     at_z2 = make_float2(at.z, at.z);
#pragma unroll 1
        for (int j = kk0; j < K / 2; j += STEP) {
          const float4 xy = bp[2 * j], zo = bp[2 * j + 1];
          const float2 dx = __fadd2_rn(at_x2, make_float2(xy.x, xy.y));
          const float2 dy = __fadd2_rn(at_y2, make_float2(xy.z, xy.w));
          const float2 dz = __fadd2_rn(at_z2, make_float2(zo.x, zo.y));
          const float2 c2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          one(2 * j, c2.x, zo.z);
          one(2 * j + 1, c2.y, zo.w);
        }
      } else {
#pragma unroll 2
        for (int k = kk0; k < K; k += STEP) {
          const float4 sh = bp[k];
          const float dx = at.x - sh.x, dy = at.y - sh.y, dz = at.z - sh.z;
          one(k, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), sh.w);
        }
      }
      if (async_rows) cp_async_wait_all();   // this thread's copies of chunk q
      __syncthreads();
      if (more) {
        if (async_rows) stage_rows_async(nxt); else stage_rows(nxt);
      }

      // ---- phase B: channel accumulation ----
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        float wv[PB];
        if constexpr (PB == 4) {
          const float4 q4 = *reinterpret_cast<const float4*>(&S.w[cur][k][pg * 4]);
          wv[0] = q4.x; wv[1] = q4.y; wv[2] = q4.z; wv[3] = q4.w;
        } else if constexpr (PB == 2) {
          const float2 q2 = *reinterpret_cast<const float2*>(&S.w[cur][k][pg * 2]);
          wv[0] = q2.x; wv[1] = q2.y;
        } else {
#pragma unroll
          for (int i = 0; i < PB; ++i) wv[i] = S.w[cur][k][pg * PB + i];
        }
        bool any = false;
#pragma unroll
        for (int i = 0; i < PB; ++i) any |= (wv[i] != 0.f);
        if (!any) continue;
        float2 w2[PB];
#pragma unroll
        for (int i = 0; i < PB; ++i) w2[i] = make_float2(wv[i], wv[i]);
#pragma unroll
        for (int q4 = 0; q4 < CB / 4; ++q4) {
          const float4 dv = *reinterpret_cast<const float4*>(&S.d[cur][k][4 * cg + 4 * NCG * q4]);
          const float2 d01 = make_float2(dv.x, dv.y), d23 = make_float2(dv.z, dv.w);
#pragma unroll
          for (int i = 0; i < PB; ++i) {
            acc[i][2 * q4] = __ffma2_rn(w2[i], d01, acc[i][2 * q4]);
            acc[i][2 * q4 + 1] = __ffma2_rn(w2[i], d23, acc[i][2 * q4 + 1]);
          }
        }
      }
    }
  }
  __syncthreads();   // the last chunk's accumulation is done with shared memory

  // ---- non-finite rows ----
  // A non-finite channel value reaches every target of a thread that some
  // of them reach (0 x NaN).  A target row (this CTA's channels) with a
  // non-finite numerator is flagged for the fix-up pass, which computes it
  // again with only the pairs inside the support (paper Eq. 1-2) and stores
  // or adds it; the row is not written here.  A sum turns non-finite when a
  // term is (or, harmlessly, on an overflow, which only sends the row to the
  // exact fix-up).
  bool row_bad[PB];
  {
    float chk[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      chk[i] = 0.f;
#pragma unroll
      for (int j = 0; j < CB / 2; ++j) chk[i] += acc[i][j].x + acc[i][j].y;
    }
    const unsigned any_bad = __syncthreads_or([&] {
      bool b = false;
#pragma unroll
      for (int i = 0; i < PB; ++i) b |= !isfinite(chk[i]);
      return b;
    }());
    if (any_bad) {
      // the NCG threads of a target group share each row: agree per row
      if (tid < kTile) S.row_nf[tid] = 0;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PB; ++i)
        if (!isfinite(chk[i])) S.row_nf[pg * PB + i] = 1;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PB; ++i) row_bad[i] = S.row_nf[pg * PB + i] != 0;
      if (tid < kTile && S.row_nf[tid] && a.tgt_perm[tile * kTile + tid] != 0xffffffffu) {
        const uint64_t e = (uint64_t)(tile * kTile + tid) * (uint64_t)n_slabs + (uint64_t)slab;
        atomicOr(&a.nf_bits[e >> 5], 1u << (e & 31));
        atomicOr(a.nf_any, 1u);
      }
    } else {
#pragma unroll
      for (int i = 0; i < PB; ++i) row_bad[i] = false;
    }
  }

  if (a.out) {
    // ---- one-shot epilogue: R = N / W (paper Eq. 3) straight into the
    // caller's [P][C] map; every slab's CTA holds all of the tile's weights
    S.wred[tid] = make_float2(ws, wc);
    if (slab == 0) {
      unsigned c = npair;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if ((tid & 31) == 0 && c && a.pairs) atomicAdd(a.pairs, (unsigned long long)c);
    }
    __syncthreads();
    if (kk0 == 0) {
      float s = 0.f, c = 0.f;
#pragma unroll
      for (int q = 0; q < STEP; ++q) {
        const float2 v = S.wred[q * kTile + p];
        const float t = s + v.x;
        const float bp2 = t - s;
        c += (s - (t - bp2)) + (v.x - bp2) + v.y;
        s = t;
      }
      S.wfin[p] = s + c;
      const uint32_t u = a.tgt_perm[slot];
      if (slab == 0 && a.out_w && u != 0xffffffffu) a.out_w[u] = s + c;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PB; ++i) {
      const int64_t sl = tile * kTile + pg * PB + i;
      const uint32_t u = a.tgt_perm[sl];
      if (u == 0xffffffffu || row_bad[i]) continue;
      const float W = S.wfin[pg * PB + i];
      float* dst = a.out + (size_t)u * C;
#pragma unroll
      for (int q = 0; q < CB / 4; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c_base + 4 * cg + 4 * NCG * q + j;
          const float2 v2 = acc[i][2 * q + (j >> 1)];
          const float v = (j & 1) ? v2.y : v2.x;
          if (c < C) dst[c] = (W > 0.f) ? v / W : __int_as_float(0x7fc00000);
        }
    }
    return;
  }

  // ---- epilogue: numerator ----
  const bool splits = a.n_split > 1;
#pragma unroll
  for (int i = 0; i < PB; ++i) {
    const int64_t sl = tile * kTile + pg * PB + i;
    if (a.tgt_perm[sl] == 0xffffffffu || row_bad[i]) continue;
    float* dst = splits ? a.part_num + ((size_t)split * a.n_slots + sl) * C
                        : a.acc_num + (size_t)sl * C;
    const bool add = a.accumulate && !splits;
#pragma unroll
    for (int q = 0; q < CB / 4; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c_base + 4 * cg + 4 * NCG * q + j;
        const float2 v2 = acc[i][2 * q + (j >> 1)];
        const float v = (j & 1) ? v2.y : v2.x;
        if (c < C) dst[c] = add ? dst[c] + v : v;
      }
  }
  // ---- epilogue: weight map and pair count (first channel slab only) ----
  if (slab != 0) return;
  S.wred[tid] = make_float2(ws, wc);
  {
    unsigned c = npair;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((tid & 31) == 0 && c && a.pairs) atomicAdd(a.pairs, (unsigned long long)c);
  }
  __syncthreads();
  if (kk0 == 0 && a.tgt_perm[slot] != 0xffffffffu) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int q = 0; q < STEP; ++q) {
      const float2 v = S.wred[q * kTile + p];
      const float t = s + v.x;
      const float bp2 = t - s;
      c += (s - (t - bp2)) + (v.x - bp2) + v.y;
      s = t;
    }
    if (splits) {
      a.part_w[(size_t)split * a.n_slots + slot] = make_float2(s, c);
      return;
    }
    float2 old = a.accumulate ? a.acc_w[slot] : make_float2(0.f, 0.f);
    const float t = old.x + s;
    const float bp2 = t - old.x;
    const float err = (old.x - (t - bp2)) + (s - bp2);
    a.acc_w[slot] = make_float2(t, old.y + c + err);
  }
}

template <int PB, int CB, int NCG, typename DT>
__global__ void __launch_bounds__((kTile / PB) * NCG) k_grid_f32(const __grid_constant__ GridArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& S = *reinterpret_cast<F32Smem<PB, CB, NCG>*>(smem_raw);
  grid_item_f32<PB, CB, NCG, DT>(a, S, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.y);
}

// Sum the candidate-split partials in split order into the accumulators.
__global__ void k_split_reduce(const float* __restrict__ part_num,
                               const float2* __restrict__ part_w,
                               const uint32_t* __restrict__ perm, int64_t n_slots, int C,
                               int n_split, int accumulate, float* __restrict__ acc_num,
                               float2* __restrict__ acc_w, const uint32_t* __restrict__ nf_bits,
                               int cpad, int n_slabs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_slots * (C + 1)) return;
  if (e < n_slots * C) {
    const int64_t sl = e / C;
    if (perm[sl] == 0xffffffffu) return;
    // a row some split flagged as non-finite is the fix-up pass's to write
    const uint64_t b = (uint64_t)sl * (uint64_t)n_slabs + (uint64_t)((e - sl * C) / cpad);
    if ((nf_bits[b >> 5] >> (b & 31)) & 1u) return;
    float v = 0.f;
    for (int z = 0; z < n_split; ++z) v += part_num[(size_t)z * n_slots * C + e];
    acc_num[e] = accumulate ? acc_num[e] + v : v;
    return;
  }
  const int64_t sl = e - n_slots * C;
  if (perm[sl] == 0xffffffffu) return;
  float s = 0.f, c = 0.f;
  for (int z = 0; z < n_split; ++z) {
    const float2 v = part_w[(size_t)z * n_slots + sl];
    const float t = s + v.x;
    const float bp = t - s;
    c += (s - (t - bp)) + (v.x - bp) + v.y;
    s = t;
  }
  float2 old = accumulate ? acc_w[sl] : make_float2(0.f, 0.f);
  const float t = old.x + s;
  const float bp = t - old.x;
  const float err = (old.x - (t - bp)) + (s - bp);
  acc_w[sl] = make_float2(t, old.y + c + err);
}

// Candidate splits for a launch: enough CTAs to fill the GPU when the
// targets form few tiles (e.g. 8,100 targets and 1e8 samples).
template <int PB, int CB, int NCG>
int splits_for(int64_t n_tiles, int C, int n_sms) {
  constexpr int NTH = (kTile / PB) * NCG;
  constexpr int CPAD = CB * NCG;
  const int64_t ctas = n_tiles * ((C + CPAD - 1) / CPAD);
  const int64_t want = (int64_t)n_sms * 1024;   // threads to fill the SMs
  int64_t s = (want + ctas * NTH - 1) / (ctas * NTH);
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

template <int PB, int CB, int NCG>
cudaError_t launch(const GridArgs& a, int64_t n_tiles, int dtype, cudaStream_t s) {
  constexpr int NTH = (kTile / PB) * NCG;
  constexpr int CPAD = CB * NCG;
  const dim3 grid((unsigned)n_tiles, (unsigned)((a.C + CPAD - 1) / CPAD), (unsigned)a.n_split);
  if (n_tiles == 0) return cudaSuccess;
  const size_t smem = sizeof(F32Smem<PB, CB, NCG>);
  if (dtype == CG_BF16) {
    auto k = k_grid_f32<PB, CB, NCG, __nv_bfloat16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTH, smem, s>>>(a);
  } else {
    auto k = k_grid_f32<PB, CB, NCG, float>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTH, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// One FP32 gridder pass: choose the candidate splits, grow the partial-sum
// scratch if needed, launch, reduce the splits, and compute the flagged
// non-finite rows again.  A one-shot output (a.out) is kept only without
// candidate splits; *direct tells whether the map was written.
template <int PB, int CB, int NCG>
cudaError_t run(cg_grid* g, GridArgs& a, int dtype, bool* direct) {
  constexpr int CPAD = CB * NCG;
  const int64_t nt = g->t64.n_tiles;
  cudaStream_t s = g->stream;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  a.n_split = splits_for<PB, CB, NCG>(nt, a.C, nsm);
  a.part_num = nullptr;
  a.part_w = nullptr;
  if (a.n_split > 1 || a.accumulate) {
    a.out = nullptr;
    a.out_w = nullptr;
  }
  if (direct) *direct = a.out != nullptr;
  if (a.n_split > 1) {
    const size_t need_n = (size_t)a.n_split * (size_t)g->n_slots * (size_t)a.C;
    const size_t need_w = (size_t)a.n_split * (size_t)g->n_slots;
    cudaError_t e;
    if (g->part_cap_num < need_n) {
      dfree(g->part_num, s);
      g->part_cap_num = 0;
      if ((e = dalloc(&g->part_num, need_n, s)) != cudaSuccess) return e;
      g->part_cap_num = need_n;
    }
    if (g->part_cap_w < need_w) {
      dfree(g->part_w, s);
      g->part_cap_w = 0;
      if ((e = dalloc(&g->part_w, need_w, s)) != cudaSuccess) return e;
      g->part_cap_w = need_w;
    }
    a.part_num = g->part_num;
    a.part_w = g->part_w;
  }
  const int n_slabs = (a.C + CPAD - 1) / CPAD;
  cudaError_t e = nonfinite_prepare(g, g->n_slots * (int64_t)n_slabs);
  if (e != cudaSuccess) return e;
  a.nf_bits = g->nf_bits;
  a.nf_any = g->nf_any;
  g->n_launches += 1;
  e = launch<PB, CB, NCG>(a, nt, dtype, s);
  if (e != cudaSuccess || nt == 0) return e;
  if (a.n_split > 1) {
    const int64_t m = g->n_slots * (int64_t)(a.C + 1);
    k_split_reduce<<<ceil_div(m, 256), 256, 0, s>>>(a.part_num, a.part_w, a.tgt_perm, g->n_slots,
                                                    a.C, a.n_split, a.accumulate, a.acc_num,
                                                    a.acc_w, a.nf_bits, CPAD, n_slabs);
    g->n_launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  NonfiniteRows rows;
  rows.tiling = &g->t64;
  rows.data = a.data;
  rows.dtype = dtype;
  rows.C = a.C;
  rows.cp = CPAD;
  rows.n_slabs = n_slabs;
  rows.mode = a.out ? 2 : (a.accumulate ? 1 : 0);
  rows.out = a.out;
  rows.acc_num = a.acc_num;
  rows.kd = a.kd;
  return nonfinite_fixup(g, rows);
}

}  // namespace

cudaError_t grid_tiles_f32(cg_grid* g, const void* data, int dtype, float* out, float* out_w,
                           bool* direct) {
  return grid_tiles_f32_to(g, data, dtype, g->acc_num, g->acc_w, g->acc_empty ? 0 : 1, 0.f, -1,
                           out, out_w, direct);
}

cudaError_t grid_tiles_f32_to(cg_grid* g, const void* data, int dtype, float* acc_num,
                              float2* acc_w, int accumulate, float dscale, int C, float* out,
                              float* out_w, bool* direct) {
  if (direct) *direct = false;
  if (C < 0) C = g->C;
  GridArgs a;
  a.out = out;
  a.out_w = out_w;
  a.tile_chi = g->t64.chi;
  a.tile_clo = g->t64.clo;
  a.tgt_a = g->t64.a;
  a.tgt_f1 = g->tgt_f1;
  a.tgt_f2 = g->tgt_f2;
  a.tgt_ll = g->tgt_ll;
  a.tgt_perm = g->tgt_perm;
  a.range_off = g->t64.range_off;
  a.range_s = g->t64.range_s;
  a.s_hi = g->s_hi;
  a.s_lo = g->s_lo;
  a.perm = g->sorted_val;
  a.sll = g->s_ll;
  a.data = data;
  a.C = C;
  const size_t esz = (dtype == CG_BF16) ? 2 : 4;
  a.vec4 = (C % 4 == 0) && ((reinterpret_cast<uintptr_t>(data) % (4 * esz)) == 0);
  a.kd = g->kdev;
  a.kd.dscale = dscale;
  a.acc_num = acc_num;
  a.acc_w = acc_w;
  a.accumulate = accumulate;
  // only the handle's own accumulation counts pairs (not the scratch passes)
  a.pairs = (dscale != 0.f || acc_num != g->acc_num) ? nullptr : g->d_pairs;
  a.tile_cand = g->t64.tile_cand;
  a.n_slots = g->n_slots;
  int cfg = g->f32_cfg;
  if (cfg < 0 || cfg >= kF32Configs || C != g->C) cfg = f32_default_config(C);
  switch (cfg) {
    case 0: return run<1, 4, 1>(g, a, dtype, direct);
    case 1: return run<1, 8, 1>(g, a, dtype, direct);
    case 2: return run<1, 8, 2>(g, a, dtype, direct);
    case 3: return run<2, 8, 4>(g, a, dtype, direct);
    case 4: return run<2, 16, 4>(g, a, dtype, direct);
    case 5: return run<4, 16, 8>(g, a, dtype, direct);
    default: return run<4, 16, 16>(g, a, dtype, direct);
  }
}

// ---------------------------------------------------------------------------
// Rows flagged as non-finite by either gridder: one CTA per (target slot,
// channel slab) bit, computed again from the tile's candidates with the FP32
// weights of pair_weight; only pairs inside the support take part, so a
// non-finite channel value reaches exactly the targets within its support
// (paper Eq. 1-2).  W itself was right (the weights are finite); the
// numerator is stored, added or (one-shot tensor-core calls) divided by W
// into the caller's map.
// ---------------------------------------------------------------------------
namespace {

struct FixArgs {
  const float4* chi;
  const float4* clo;
  const float4* ta;
  const int64_t* range_off;
  const int2* range_s;
  int T;                  // targets per tile of the tiling the rows belong to
  const float4* f1;
  const float4* f2;
  const double2* tll;
  const float4* s_hi;
  const float4* s_lo;
  const uint32_t* perm;
  const double2* sll;
  KernelDev kd;
  const void* data;
  int bf16;
  int C, cp, n_slabs, mode;
  float* out;
  float* acc_num;
  const uint32_t* perm_t;
  uint32_t* bits;
  const uint32_t* any;
  int64_t n_words;
};

constexpr int kFixThreads = 256;

__device__ __forceinline__ float fix_load(const FixArgs& a, size_t i) {
  return a.bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.data)[i])
                : static_cast<const float*>(a.data)[i];
}

struct FixShared {
  float w[kFixThreads];
  uint32_t idx[kFixThreads];
  double wsum[kFixThreads];
  uint32_t word;
};

// The flagged rows of bitmap word wd (the whole CTA; clears the word).
__device__ __forceinline__ void fix_word(const FixArgs& a, int64_t wd, FixShared& F) {
  const int tid = threadIdx.x;
  __syncthreads();
  if (tid == 0) F.word = a.bits[wd];
  __syncthreads();
  uint32_t bits = F.word;
  if (!bits) return;
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    const int64_t e = wd * 32 + b;
    const int64_t slot = e / a.n_slabs;
    const int slab = (int)(e % a.n_slabs);
    const int64_t tile = slot / a.T;
    const float4 at = a.ta[slot];
    float4 f1 = make_float4(0.f, 0.f, 0.f, 0.f), f2 = f1;
    if (a.kd.type == CG_GAUSS2D) {
      f1 = a.f1[slot];
      f2 = a.f2[slot];
    }
    const float4 chi = a.chi[tile], clo = a.clo[tile];
    const int c = slab * a.cp + tid;
    const bool mine = tid < a.cp && c < a.C;
    float acc = 0.f;
    double wsum = 0.0;
    for (int64_t r = a.range_off[tile]; r < a.range_off[tile + 1]; ++r) {
      const int2 rg = a.range_s[r];
      for (int j0 = rg.x; j0 < rg.y; j0 += kFixThreads) {
        __syncthreads();
        const int pos = j0 + tid;
        float w = -0.f;
        uint32_t idx = 0;
        if (pos < rg.y) {
          const float4 h = a.s_hi[pos], l = a.s_lo[pos];
          const float4 sh = make_float4(df_diff(h.x, l.x, chi.x, clo.x),
                                        df_diff(h.y, l.y, chi.y, clo.y),
                                        df_diff(h.z, l.z, chi.z, clo.z), h.w);
          idx = a.perm[pos];
          bool in;
          w = pair_weight(a.kd, at, f1, f2, sh, a.tll[slot], a.sll, idx, in);
          if (in) wsum += (double)w;
        }
        F.w[tid] = w;
        F.idx[tid] = idx;
        __syncthreads();
        const int n = min(kFixThreads, rg.y - j0);
        if (mine)
          for (int k = 0; k < n; ++k)
            if (takes_part(F.w[k])) acc = fmaf(F.w[k], fix_load(a, (size_t)F.idx[k] * a.C + c), acc);
      }
    }
    double W = 0.0;
    if (a.mode == 2) {
      F.wsum[tid] = wsum;
      __syncthreads();
      for (int o = kFixThreads / 2; o > 0; o >>= 1) {
        if (tid < o) F.wsum[tid] += F.wsum[tid + o];
        __syncthreads();
      }
      W = F.wsum[0];
    }
    if (mine) {
      if (a.mode == 2) {
        const uint32_t user = a.perm_t[slot];
        if (user != 0xffffffffu)
          a.out[(size_t)user * a.C + c] = (W > 0.0) ? (float)((double)acc / W) : __int_as_float(0x7fc00000);
      } else if (a.mode == 1) {
        a.acc_num[(size_t)slot * a.C + c] += acc;
      } else {
        a.acc_num[(size_t)slot * a.C + c] = acc;
      }
    }
  }
  __syncthreads();
  if (tid == 0) a.bits[wd] = 0u;
}

__global__ void __launch_bounds__(kFixThreads) k_nonfinite_fixup(FixArgs a) {
  __shared__ FixShared F;
  if (*a.any == 0u) return;   // the common case: nothing flagged
  for (int64_t wd = blockIdx.x; wd < a.n_words; wd += gridDim.x) fix_word(a, wd, F);
}

}  // namespace

cudaError_t nonfinite_prepare(cg_grid* g, int64_t n_bits) {
  const size_t words = (size_t)((n_bits + 31) / 32);
  if (g->nf_words < words) {
    // zero when allocated; every fix-up pass clears the bits it served
    dfree(g->nf_bits, g->stream);
    g->nf_words = 0;
    cudaError_t e = dalloc(&g->nf_bits, words, g->stream);
    if (e == cudaSuccess && !g->nf_any) e = dalloc(&g->nf_any, 1, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->nf_bits, 0, words * sizeof(uint32_t), g->stream);
    if (e != cudaSuccess) return e;
    g->nf_words = words;
  }
  return cudaMemsetAsync(g->nf_any, 0, sizeof(uint32_t), g->stream);
}

cudaError_t nonfinite_fixup(cg_grid* g, const NonfiniteRows& j) {
  FixArgs a;
  const Tiling& t = *j.tiling;
  a.chi = t.chi;
  a.clo = t.clo;
  a.ta = t.a;
  a.range_off = t.range_off;
  a.range_s = t.range_s;
  a.T = t.T;
  a.f1 = g->tgt_f1;
  a.f2 = g->tgt_f2;
  a.tll = g->tgt_ll;
  a.s_hi = g->s_hi;
  a.s_lo = g->s_lo;
  a.perm = g->sorted_val;
  a.sll = g->s_ll;
  a.kd = j.kd;
  a.data = j.data;
  a.bf16 = j.dtype == CG_BF16;
  a.C = j.C;
  a.cp = j.cp;
  a.n_slabs = j.n_slabs;
  a.mode = j.mode;
  a.out = j.out;
  a.acc_num = j.acc_num;
  a.perm_t = g->tgt_perm;
  a.bits = g->nf_bits;
  a.any = g->nf_any;
  a.n_words = (int64_t)((g->n_slots * (int64_t)j.n_slabs + 31) / 32);
  if (j.cp > kFixThreads || a.n_words > (int64_t)g->nf_words) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  k_nonfinite_fixup<<<(unsigned)nsm, kFixThreads, 0, g->stream>>>(a);
  g->n_launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused batches: one FP32 gridder launch for the items of all jobs.
// ---------------------------------------------------------------------------
namespace {

constexpr int kMultiBins = 256;
constexpr int kOrderCta = 1024;

// Largest j with off[j] <= x (off[0] = 0, off non-decreasing, x < off[n]).
__device__ __forceinline__ int find_job(const int64_t* __restrict__ off, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct ItemPos {
  int job;
  int64_t tile;
  int slab, split, n_slabs;
};

__device__ __forceinline__ ItemPos decode_item(const F32Multi& m, int64_t it) {
  ItemPos q;
  q.job = find_job(m.item_off, m.n_jobs, it);
  const F32MultiJob& J = m.jobs[q.job];
  const int64_t local = it - m.item_off[q.job];
  const int ns = J.a.n_split, nb = J.n_slabs;
  q.n_slabs = nb;
  q.tile = local / ((int64_t)nb * ns);
  const int r = (int)(local - q.tile * nb * ns);
  q.slab = r / ns;
  q.split = r % ns;
  return q;
}

// Decreasing estimated cost (weights of the tile's share of candidates plus
// its channel work), in log-spaced bins.
__device__ __forceinline__ int multi_bin(const F32Multi& m, int64_t it) {
  const ItemPos q = decode_item(m, it);
  const F32MultiJob& J = m.jobs[q.job];
  const int ns = J.a.n_split;
  const float cand = (float)((J.a.tile_cand[q.tile] + ns - 1) / ns);
  const float cost = cand * (float)(kTile + J.pad);
  const int b = (int)(8.f * __log2f(1.f + cost));
  return kMultiBins - 1 - min(max(b, 0), kMultiBins - 1);
}

// One CTA: the queue order (counting sort by cost bin), and the queue head
// and the non-finite flag cleared for the gridder launch that follows.
__global__ void __launch_bounds__(kOrderCta) k_multi_order(const __grid_constant__ F32Multi m) {
  __shared__ int32_t cnt[kMultiBins];
  __shared__ int32_t wsum[kOrderCta / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    *m.head = 0u;
    *m.nf_any = 0u;
  }
  for (int i = tid; i < kMultiBins; i += kOrderCta) cnt[i] = 0;
  __syncthreads();
  for (int64_t it = tid; it < m.n_items; it += kOrderCta) atomicAdd(&cnt[multi_bin(m, it)], 1);
  __syncthreads();
  // exclusive scan of the bins (one per thread of the first kMultiBins)
  const int v = tid < kMultiBins ? cnt[tid] : 0;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  if (tid < kMultiBins) cnt[tid] = incl - v + (warp > 0 ? wsum[warp - 1] : 0);
  __syncthreads();
  for (int64_t it = tid; it < m.n_items; it += kOrderCta) {
    const int pos = atomicAdd(&cnt[multi_bin(m, it)], 1);
    m.order[pos] = (int32_t)it;
  }
}

template <int PB, int CB, int NCG>
__device__ __forceinline__ void multi_item(const GridArgs& a, unsigned char* raw, int dtype,
                                           const ItemPos& q) {
  auto& S = *reinterpret_cast<F32Smem<PB, CB, NCG>*>(raw);
  if (dtype == CG_BF16)
    grid_item_f32<PB, CB, NCG, __nv_bfloat16>(a, S, q.tile, q.slab, q.split, q.n_slabs);
  else
    grid_item_f32<PB, CB, NCG, float>(a, S, q.tile, q.slab, q.split, q.n_slabs);
}

// The gridder launch carries every job's arguments in its parameter space, so
// that the items read them as constant operands (like a one-job launch).
struct MultiLaunch {
  F32Multi m;
  GridArgs ga[kF32MultiMaxJobs];
};

// Persistent CTAs take items from the queue until it is empty.  One kernel
// per register-blocking shape of the one-job gridder (the jobs of a launch
// share it), held to the one-job kernel's CTAs per SM (MINB); as many CTAs as
// fit on the GPU.
template <int PB, int CB, int NCG, int MINB>
__global__ void __launch_bounds__((kTile / PB) * NCG, MINB)
    k_grid_f32_multi(const __grid_constant__ MultiLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const F32Multi& m = L.m;
  __shared__ int64_t s_item;
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_stop = 0;
    if (m.hold) {
      // testing hook: wait for a word that nothing sets; the wait runs out
      // and the CTA leaves without taking an item
      const long long t0 = clock64();
      while (*((volatile const int*)m.hold) == 0 && clock64() - t0 < m.hold_cycles) __nanosleep(1000);
      if (*((volatile const int*)m.hold) == 0) {
        set_error(m.err, ERR_TIMEOUT);
        s_stop = 1;
      }
    }
  }
  __syncthreads();
  if (s_stop) return;
  for (;;) {
    if (tid == 0) {
      const unsigned q = atomicAdd(m.head, 1u);
      s_item = (int64_t)q < m.n_items ? (int64_t)m.order[q] : -1;
    }
    __syncthreads();
    const int64_t it = s_item;
    if (it < 0) break;
    const ItemPos q = decode_item(m, it);
    const int dtype = m.jobs[q.job].dtype;
    const GridArgs& ja = L.ga[__shfl_sync(0xffffffffu, q.job, 0)];
    multi_item<PB, CB, NCG>(ja, smem_raw, dtype, q);
    __syncthreads();   // the item is done with s_item and shared memory
  }
}

// Candidate-split partials of every split job, in split order, into its
// accumulators; rows flagged as non-finite are left to the fix-up.  CTA b
// serves kMultiRedElems values of the job whose CTA range holds b: the
// numerator [slots][C], then the weight map [slots].
__global__ void __launch_bounds__(kMultiRedElems) k_multi_reduce(const __grid_constant__ F32Multi m) {
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = find_job(m.red_blk, m.n_jobs, blockIdx.x);
  __syncthreads();
  const int job = s_job;
  const F32MultiJob& J = m.jobs[job];
  const int ns = J.a.n_split;
  const int C = J.a.C;
  const int64_t n_slots = J.a.n_slots;
  const int64_t le = (int64_t)(blockIdx.x - m.red_blk[job]) * kMultiRedElems + threadIdx.x;
  if (le < n_slots * C) {
    const int64_t sl = le / C;
    if (J.a.tgt_perm[sl] == 0xffffffffu) return;
    const uint64_t b = (uint64_t)sl * (uint64_t)J.n_slabs + (uint64_t)((le - sl * C) / J.pad);
    if ((J.a.nf_bits[b >> 5] >> (b & 31)) & 1u) return;
    float v = 0.f;
    for (int z = 0; z < ns; ++z) v += J.a.part_num[(size_t)z * n_slots * C + le];
    J.a.acc_num[le] = v;
    return;
  }
  const int64_t sl = le - n_slots * C;
  if (sl >= n_slots || J.a.tgt_perm[sl] == 0xffffffffu) return;
  float s = 0.f, c = 0.f;
  for (int z = 0; z < ns; ++z) {
    const float2 v = J.a.part_w[(size_t)z * n_slots + sl];
    const float t = s + v.x;
    const float bp = t - s;
    c += (s - (t - bp)) + (v.x - bp) + v.y;
    s = t;
  }
  J.a.acc_w[sl] = make_float2(s, c);
}

// The flagged rows of all jobs (bitmap words of all jobs, grid-stride).
__global__ void __launch_bounds__(kFixThreads) k_multi_fixup(const __grid_constant__ F32Multi m) {
  __shared__ FixShared F;
  if (*m.nf_any == 0u) return;
  for (int64_t gw = blockIdx.x; gw < m.n_words; gw += gridDim.x) {
    const int job = find_job(m.word_off, m.n_jobs, gw);
    const F32MultiJob& J = m.jobs[job];
    const int64_t wd = gw - m.word_off[job];
    if (J.a.nf_bits[wd] == 0u) continue;   // the same word for every thread
    FixArgs f;
    f.chi = J.a.tile_chi;
    f.clo = J.a.tile_clo;
    f.ta = J.a.tgt_a;
    f.range_off = J.a.range_off;
    f.range_s = J.a.range_s;
    f.T = kTile;
    f.f1 = J.a.tgt_f1;
    f.f2 = J.a.tgt_f2;
    f.tll = J.a.tgt_ll;
    f.s_hi = J.a.s_hi;
    f.s_lo = J.a.s_lo;
    f.perm = J.a.perm;
    f.sll = J.a.sll;
    f.kd = J.a.kd;
    f.data = J.a.data;
    f.bf16 = J.dtype == CG_BF16;
    f.C = J.a.C;
    f.cp = J.pad;
    f.n_slabs = J.n_slabs;
    f.mode = J.a.out ? 2 : 0;
    f.out = J.a.out;
    f.acc_num = J.a.acc_num;
    f.perm_t = J.a.tgt_perm;
    f.bits = J.a.nf_bits;
    f.any = m.nf_any;
    f.n_words = 0;
    fix_word(f, wd, F);
  }
}

// Eq. 3 for every job: R = N / W (NaN where W = 0) in the caller's layout.
// CTA b serves kMultiFinElems numerator values of the job whose CTA range
// holds b, four consecutive channels of one target per thread where the
// map allows 16-byte rows.
__global__ void __launch_bounds__(256) k_multi_finalize(const __grid_constant__ F32Multi m) {
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = find_job(m.fin_blk, m.n_jobs, blockIdx.x);
  __syncthreads();
  const int job = s_job;
  const F32MultiJob& J = m.jobs[job];
  const F32Multi::Out o = m.outs[job];
  const int C = J.a.C;
  const int64_t n = J.a.n_slots * C;
  const int64_t base = (int64_t)(blockIdx.x - m.fin_blk[job]) * kMultiFinElems;
  if (o.vec4) {
    const int64_t e = base + 4 * (int64_t)threadIdx.x;
    if (e >= n) return;
    const int64_t slot = e / C;
    const int c = (int)(e - slot * C);
    const uint32_t u = J.a.tgt_perm[slot];
    if (u == 0xffffffffu) return;
    const float2 w2 = J.a.acc_w[slot];
    const float W = w2.x + w2.y;
    const float4 v = *reinterpret_cast<const float4*>(J.a.acc_num + e);
    float4 r;
    if (W > 0.f) {
      r = make_float4(v.x / W, v.y / W, v.z / W, v.w / W);
    } else {
      const float q = __int_as_float(0x7fc00000);
      r = make_float4(q, q, q, q);
    }
    *reinterpret_cast<float4*>(o.out + (size_t)u * C + c) = r;
    if (o.out_w && c == 0) o.out_w[u] = W;
    return;
  }
  for (int r = 0; r < kMultiFinElems / 256; ++r) {
    const int64_t e = base + r * 256 + threadIdx.x;
    if (e >= n) return;
    const int64_t slot = e / C;
    const int c = (int)(e - slot * C);
    const uint32_t u = J.a.tgt_perm[slot];
    if (u == 0xffffffffu) continue;
    const float2 w2 = J.a.acc_w[slot];
    const float W = w2.x + w2.y;
    const float v = (W > 0.f) ? J.a.acc_num[e] / W : __int_as_float(0x7fc00000);
    if (o.channel_major) o.out[(size_t)c * o.P + u] = v;
    else o.out[(size_t)u * C + c] = v;
    if (o.out_w && c == 0) o.out_w[u] = W;
  }
}

template <int PB, int CB, int NCG, int MINB>
cudaError_t launch_multi(const MultiLaunch& L, int nsm, cudaStream_t s) {
  constexpr int NTH = (kTile / PB) * NCG;
  auto k = k_grid_f32_multi<PB, CB, NCG, MINB>;
  const size_t smem = sizeof(F32Smem<PB, CB, NCG>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTH, smem);
  if (e != cudaSuccess) return e;
  const int64_t ctas = std::min<int64_t>((int64_t)std::max(1, per_sm) * nsm, L.m.n_items);
  k<<<(unsigned)ctas, NTH, smem, s>>>(L);
  return cudaGetLastError();
}

}  // namespace

int f32_multi_shape(int C) { return f32_default_config(C); }

int f32_multi_cpad(int shape) {
  static const int cp[kF32MultiShapes] = {4, 8, 16, 32, 64, 128, 256};
  return cp[shape < 0 ? 0 : (shape >= kF32MultiShapes ? kF32MultiShapes - 1 : shape)];
}

cudaError_t grid_f32_multi(const F32Multi& m, cudaStream_t s, int64_t* launches) {
  if (m.n_items <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (m.n_jobs > kF32MultiMaxJobs || !m.hjobs) return cudaErrorInvalidValue;
  static thread_local MultiLaunch L;   // large: not on the stack (the launch copies it)
  L.m = m;
  for (int j = 0; j < m.n_jobs; ++j) L.ga[j] = m.hjobs[j].a;
  k_multi_order<<<1, kOrderCta, 0, s>>>(m);
  cudaError_t e;
  switch (m.shape) {
    case 0: e = launch_multi<1, 4, 1, 12>(L, nsm, s); break;
    case 1: e = launch_multi<1, 8, 1, 10>(L, nsm, s); break;
    case 2: e = launch_multi<1, 8, 2, 6>(L, nsm, s); break;
    case 3: e = launch_multi<2, 8, 4, 5>(L, nsm, s); break;
    case 4: e = launch_multi<2, 16, 4, 4>(L, nsm, s); break;
    case 5: e = launch_multi<4, 16, 8, 3>(L, nsm, s); break;
    default: e = launch_multi<4, 16, 16, 2>(L, nsm, s); break;
  }
  if (e != cudaSuccess) return e;
  int64_t n = 2;   // order, gridder
  if (m.n_red_blk > 0) {
    k_multi_reduce<<<(unsigned)m.n_red_blk, kMultiRedElems, 0, s>>>(m);
    ++n;
  }
  k_multi_fixup<<<(unsigned)nsm, kFixThreads, 0, s>>>(m);
  if (m.n_fin_blk > 0) {
    // only jobs whose maps the gridder did not write (splits, channel-major)
    k_multi_finalize<<<(unsigned)m.n_fin_blk, 256, 0, s>>>(m);
    ++n;
  }
  if (launches) *launches += n + 1;
  return cudaGetLastError();
}

// Register-blocking shapes of the FP32 gridder, (targets x channels per
// thread in phase B, channel groups): 0 <1,4,1> 1 <1,8,1> 2 <1,8,2>
// 3 <2,8,4> 4 <2,16,4> 5 <4,16,8> 6 <4,16,16>; a CTA covers CB * NCG channels
// of its tile, more channels take more CTAs.  The default follows C.
int f32_default_config(int C) {
  if (C <= 4) return 0;
  if (C <= 8) return 1;
  if (C <= 16) return 2;
  if (C <= 32) return 3;
  if (C <= 64) return 4;
  if (C <= 128) return 5;
  return 6;
}

}  // namespace cg
