// k_grid_tc.cu -- tile gridder, BF16 tensor-core form (paper Eq. 1-3).
//
// For a tile of 128 targets and a chunk of 32 candidate samples the kernel
// evaluates the weight matrix A[p][k] = omega_k w(p, k) (BF16) on the CUDA
// cores and accumulates D[p][c] += sum_k A[p][k] B[k][c] with B the samples'
// BF16 channel rows, on the tcgen05 tensor cores with FP32 accumulators in
// tensor memory (TMEM):
//
//   M = 128 targets (TMEM lanes), N = channels of one slab (<= 256, TMEM
//   columns), K = candidates, two K = 16 MMAs per chunk.
//
// Operands: A lives in TMEM (written with tcgen05.st by the thread that owns
// the target row, so the weights never touch shared memory).  In the default
// (split) form every weight is stored as w_hi + w_lo, two BF16 numbers
// (~16 significant bits), and each K step issues one MMA per half against
// the same B; the fast form keeps only w_hi (8 significant bits).  B is the
// MN-major SW128 canonical layout (atoms of 8 candidates x 64 channels, the
// 16-byte pieces of a 128-byte row permuted by the row index; LBO = 4 KB
// between channel blocks, SBO = 1 KB between candidate groups), filled from
// the caller's [N][C] rows by the Tensor Memory Accelerator: one
// cp.async.bulk.tensor tile::gather4 moves four arbitrary sample rows x 64
// channels with 128-byte swizzling, straight into that layout; padding
// candidates point past the last row and arrive as zeros.  A warp issues its
// lanes' gathers one after another (~40 ns each), so the copy rate grows
// with the number of issuing warps (measured: ~1.9 TB/s over the chip with
// one warp per SM, ~13 TB/s from L2 with eight); hence eight producer warps.
//
// Warp roles (persistent CTA, static round-robin over (tile, slab) items):
//   warps 0-7   weights: warp w handles target rows 32 (w % 4) .. + 31 (one
//               TMEM lane quarter, a compact 32-target k-d leaf) and
//               candidates 16 (w / 4) .. + 15 of every chunk, as two groups of
//               8; a group that cannot reach the quarter (disc of radius
//               quarter radius + r) is skipped; the FP32 arithmetic runs on
//               pairs of candidates with the packed f32x2 instructions;
//               weight-map partial sums (compensated) per item;
//   warps 8-15  producers (chunk q belongs to warp q % 8, which owns stage
//               q % 8): locate the chunk's candidates in the tile's sample
//               ranges, write their tile-relative vectors, gather their data
//               rows; the next own chunk's loads are issued before waiting
//               for the stage to be free;
//   warps 16-19 epilogue (one per TMEM lane quarter): W from the weight
//               warps' partials, D -> registers -> R = N / W (or the
//               accumulators), then D is released to the next item;
//   warp 20     MMA issue (one lane) and tcgen05.commit.
// Every mbarrier wait is bounded; on time-out the kernel records
// ERR_TIMEOUT, stops issuing work, waits for its own MMAs and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>

#include "cg_common.cuh"
#include "cg_cut.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

constexpr int kT = kTile2;          // targets per tile = MMA M
constexpr int kK = 32;              // candidates per chunk
constexpr int kWW = 8;              // weight warps (2 per TMEM lane quarter)
constexpr int kGPW = 2;             // groups of 8 candidates per weight warp and chunk
static_assert(kGPW * 8 * (kWW / 4) == 32, "weight warps cover a chunk");
constexpr int kNP = 8;              // producer warps (chunk q goes to warp q % kNP)
constexpr int kEW = 4;              // epilogue warps (one per TMEM lane quarter)
constexpr int kThreads = (kWW + kNP + kEW + 1) * 32;
constexpr int kProdWarp = kWW;      // first producer warp
constexpr int kEpiWarp = kWW + kNP; // first epilogue warp
constexpr int kMmaWarp = kWW + kNP + kEW;
constexpr int kEpiPitch = 36;       // floats per row of an epilogue tile (32 + pad)
constexpr int kNS = 8;             // pipeline stages (one per producer warp)
constexpr int kMaxStages = kNS;
// a wait gives up after ~1 s of SM clock (or at once after another role gave up)
constexpr long long kWaitCycles = 2000000000LL;
// longest single suspension inside a wait (ns); the time-out is checked between
constexpr uint32_t kSuspendNs = 20000;

struct TcArgs {
  const float4* chi;
  const float4* clo;
  const float4* ta;
  const float4* subf;   // per tile x quarter: centre rel. to the tile centre, chord radius
  const int64_t* range_off;
  const int2* range_s;
  const int32_t* range_c;
  const int32_t* tile_cand;
  const int32_t* order;  // items by decreasing cost (null: round-robin over item indices)
  int64_t n_tiles;
  const float4* f1;
  const float4* f2;
  const double2* tll;
  const uint32_t* perm_t;
  const float4* s_hi;
  const float4* s_lo;
  const uint32_t* sperm;
  const double2* sll;   // FP64 lon/lat of each sample (input order, degrees)
  const __nv_bfloat16* data;
  int C;
  int cp;        // padded channels per slab (multiple of 64, <= 256)
  int n_slabs;
  int split;     // 1: weights as hi + lo BF16 pairs (two MMAs per K step)
  uint32_t tmem_cols;
  KernelDev kd;
  int mode;      // 0 store, 1 add, 2 one-shot normalised output
  float* acc_num;
  float2* acc_w;
  float* out;
  float* out_w;
  int n_rows;    // samples (rows of the data tensor)
  int64_t P;
  int64_t n_slots;
  unsigned long long* pairs;
  unsigned* err;
  uint32_t* nf_bits;    // (slot, slab) rows with a non-finite numerator
  uint32_t* nf_any;
  const int* hold;      // cg_debug_hold: a word nothing sets (null: no hold)
  long long hold_cycles;
};

struct Smem {
  uint8_t* B;          // ns stages of cp * 64 bytes
  float* cand;         // ns x kK/2 pairs x 8: (x0 x1 y0 y1) (z0 z1 l0 l1), l = log2 omega + e_mid
  float* reach;        // ns x 4 quarters x kK: squared chord to the quarter centre
  uint32_t* cidx;      // ns x kK: row of the caller's arrays
  float2* wpart;       // 2 buffers x (kWW / 4) groups x kT partial weight sums
  float* epi;          // kEW x 32 x kEpiPitch: epilogue transpose tiles
  uint64_t* full;      // ns: data rows landed (TMA transaction bytes)
  uint64_t* cfull;     // ns: candidate vectors written
  uint64_t* afull;     // ns: weights in TMEM
  uint64_t* empty;     // ns: MMAs of the stage done
  uint64_t* dfull;     // the item's MMAs are complete (D ready)
  uint64_t* dempty;    // the epilogue has drained D
  uint64_t* fin;
  uint64_t* wfull;     // 2: the weight warps' W partials of an item are written
  uint64_t* wempty;    // 2: the epilogue has read them
  uint32_t* tmem_base;
  int* abort_flag;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(su32(b))
               : "memory");
}

// Bounded wait for the phase with the given parity: false on time-out or
// when another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity,
                                          volatile int* abort_flag) {
  const uint32_t a = su32(b);
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    // the suspend-time hint lets the warp sleep until the phase completes
    // (or the hint expires) instead of re-issuing the test
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if ((it & 3u) == 3u) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kWaitCycles) return false;
    }
  }
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(addr, lbo, sbo) | ((uint64_t)2 << 61);  // layout: 128-byte swizzle
}

// Item k of this CTA's sequence, -1 past its end.  With an order (round k
// of the schedule is a wave of G spatially consecutive items, dealt to the G
// CTAs by k_item_waves), CTA b takes order[k G + b]; without one, items b,
// b + G, b + 2 G, ...
__device__ __forceinline__ int64_t item_at(const TcArgs& a, int64_t n_items, int64_t k) {
  const int64_t G = gridDim.x;
  const int64_t pos = (int64_t)blockIdx.x + k * G;
  if (!a.order) return pos < n_items ? pos : -1;
  const int64_t waves = (n_items + G - 1) / G;
  return pos < waves * G ? (int64_t)a.order[pos] : -1;
}

__device__ __forceinline__ int chunks_of(const TcArgs& a, int64_t item) {
  return (a.tile_cand[item / a.n_slabs] + kK - 1) / kK;
}

// What a producer lane needs to stage one chunk; loaded one own chunk ahead.
struct Fetch {
  int64_t tile;
  int c_base;
  int pos;            // sorted sample position of this lane's candidate (-1: padding)
  float4 h, l;        // its double-float unit vector (h.w = omega)
  uint32_t idx;       // its row in the caller's arrays
  float4 chi, clo;    // tile centre (double-float)
  float4 sq[4];       // quarter centres relative to the tile centre
};

// Candidates 32 ch .. 32 ch + 31 of the tile of `item`: the first range whose
// cumulative count covers 32 ch, then a walk through the following ranges
// held in lanes.
__device__ __forceinline__ void fetch_chunk(const TcArgs& a, int64_t item, int ch, int lane,
                                            Fetch& f) {
  const int64_t tile = item / a.n_slabs;
  f.tile = tile;
  f.c_base = (int)(item % a.n_slabs) * a.cp;
  const int64_t r0 = a.range_off[tile], r1 = a.range_off[tile + 1];
  const int c0 = ch * kK;
  // number of ranges with cum <= c0 (cum is non-decreasing within the tile)
  int64_t cnt = 0;
  for (int64_t b = r0; b < r1; b += 32) {
    const int64_t r = b + lane;
    const bool le = (r < r1) && a.range_c[r] <= c0;
    const unsigned m = __ballot_sync(0xffffffffu, le);
    cnt += __popc(m);
    if (m != 0xffffffffu) break;
  }
  int64_t wbase = r0 + cnt - 1;   // range holding candidate c0
  int2 wr_lane = make_int2(0, 0);
  int32_t c_first = 0;
  if (wbase + lane < r1) wr_lane = a.range_s[wbase + lane];
  if (lane == 0 && wbase < r1) c_first = a.range_c[wbase];
  int off = c0 - __shfl_sync(0xffffffffu, c_first, 0);
  int wr = 0, filled = 0, pos = -1;
  while (filled < kK) {
    if (wr == 32) {
      wbase += 32;
      wr = 0;
      if (wbase >= r1) break;
      wr_lane = (wbase + lane < r1) ? a.range_s[wbase + lane] : make_int2(0, 0);
    }
    if (wbase + wr >= r1) break;
    const int rs = __shfl_sync(0xffffffffu, wr_lane.x, wr);
    const int re = __shfl_sync(0xffffffffu, wr_lane.y, wr);
    const int avail = re - rs - off;
    const int take = min(kK - filled, avail);
    if (take > 0) {
      if (lane >= filled && lane < filled + take) pos = rs + off + (lane - filled);
      filled += take;
      off += take;
    }
    if (off >= re - rs) {
      ++wr;
      off = 0;
    }
  }
  f.pos = pos;
  f.idx = 0xffffffffu;
  if (pos >= 0) {
    f.h = a.s_hi[pos];
    f.l = a.s_lo[pos];
    f.idx = a.sperm[pos];
  }
  f.chi = a.chi[tile];
  f.clo = a.clo[tile];
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) f.sq[qq] = a.subf[tile * 4 + qq];
}

// Next own chunk: global chunk q + kNP, i.e. kNP chunks further along the
// CTA's sequence of (item, chunk) pairs; item k of the sequence is `item`.
__device__ __forceinline__ void advance(const TcArgs& a, int64_t n_items, int64_t& k,
                                        int64_t& item, int& ch, int& nch, int step) {
  ch += step;
  while (item >= 0 && ch >= nch) {
    ch -= nch;
    item = item_at(a, n_items, ++k);
    nch = (item >= 0) ? chunks_of(a, item) : 0;
  }
}

// Constants of the weight evaluation (per kernel launch).  The squared chord
// is carried as x = c2 - mid, mid the centre of the guard band [c2_in,
// c2_out] (the FP32 sum starts from -mid, so this costs nothing): x <= hw is
// the support cut and |x| <= hw finds the pairs inside the band.  With
// c2 = x + mid the series exponent (Eq. 3 with d^2 = c2 (1 + c2 / 12))
//   q1 c2 + q2 c2^2 + log2 omega = x (q1x + q2 x) + (log2 omega + e_mid)
// with q1x = q1 + 2 q2 mid, e_mid = q1 mid + q2 mid^2; the producers store
// log2 omega + e_mid with each candidate (e_mid = 0 for the other forms).
struct PairConst {
  float2 nmid;               // (-mid, -mid)
  float2 q1x, q2;            // series form, both lanes
  float2 q1, q4;             // exponent coefficients (log2 e folded in)
  float2 mid2;               // (mid, mid)
  float mid, hw;             // band centre and half-width (chord^2)
  float e_mid;
  float inv_a;               // CG_TSINC: 1 / a (rad^-1)
};

template <int KT, bool BIG>
__device__ __forceinline__ PairConst make_pair_const(const KernelDev& kd) {
  PairConst P;
  const float mid = 0.5f * (kd.c2_in + kd.c2_out);
  P.mid = mid;
  P.hw = 0.5f * (kd.c2_out - kd.c2_in);     // exact: the two are within 2x
  P.nmid = make_float2(-mid, -mid);
  P.mid2 = make_float2(mid, mid);
  const double q1 = kd.k1, q2 = (double)kd.k1 / 12.0, m = mid;
  const bool series = KT == CG_GAUSS1D && !BIG;
  const float q1x = series ? (float)(q1 + 2.0 * q2 * m) : kd.k1;
  P.q1x = make_float2(q1x, q1x);
  P.q2 = make_float2((float)q2, (float)q2);
  P.q1 = make_float2(kd.k1, kd.k1);
  P.q4 = make_float2(kd.k2, kd.k2);
  P.e_mid = series ? (float)(q1 * m + q2 * m * m) : 0.f;
  P.inv_a = kd.inv_a;
  return P;
}

// Per-target constants: the negated tile-relative vector and (elliptical
// form) the major / minor axis directions, each duplicated for both lanes of
// a packed pair.
struct TgtConst {
  float2 nx, ny, nz;
  float2 f1x, f1y, f1z, f2x, f2y, f2z;
};

// x = c2 - mid of one candidate of a pair block, in the same operation order
// as the packed evaluation (so both give the same bits).
__device__ __forceinline__ float pair_x(const float* blk, int h, const TgtConst& T, float nmid) {
  const float dx = blk[h] + T.nx.x, dy = blk[2 + h] + T.ny.x, dz = blk[4 + h] + T.nz.x;
  return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, nmid)));
}

// Candidates 0 .. n-1 of a group whose x lies in the guard band: the support
// cut is decided again from the input coordinates (pair_inside).  Returns the
// mask of those that lie outside the support after all.  Rare; kept out of
// line so that the common path does not carry its registers.
__device__ __noinline__ uint32_t band_fixup(const float* cand, const uint32_t* cidx, int n,
                                            TgtConst T, float nmid, float hw,
                                            const double2* tll, const double2* sll,
                                            int64_t slot, const KernelDev& kd) {
  uint32_t kill = 0;
  for (int k = 0; k < n; ++k) {
    const float x = pair_x(cand + 8 * (k >> 1), k & 1, T, nmid);
    if (fabsf(x) <= hw &&
        !pair_inside(tll[slot], sll[cidx[k]], kd.c2r_hi, kd.c2r_lo, kd.c2r_tol, kd.r_rad))
      kill |= 1u << k;
  }
  return kill;
}

// N weights omega w(p, k) of this thread's target against the candidates of
// one group (N / 2 pair blocks) into w[], zero beyond the support; np counts
// the pairs with d <= r.
template <int N, int KT, bool BIG>
__device__ __forceinline__ void eval_group(const float* cand, const uint32_t* cidx,
                                           const TgtConst& T, const PairConst& P,
                                           const TcArgs& a, int64_t slot, float* w,
                                           unsigned& np) {
  float bm = INFINITY;     // smallest |x| of this thread's pairs
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    const float4 xy = *reinterpret_cast<const float4*>(cand + 8 * j);
    const float4 zl = *reinterpret_cast<const float4*>(cand + 8 * j + 4);
    const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), T.nx);
    const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), T.ny);
    const float2 dz = __fadd2_rn(make_float2(zl.x, zl.y), T.nz);
    const float2 x = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, P.nmid)));
    const float2 lw = make_float2(zl.z, zl.w);
    float2 e;
    float2 sf = make_float2(1.f, 1.f);   // the tapered sinc's sinc factor
    if (KT == CG_TSINC) {
      const float2 c2 = __fadd2_rn(x, P.mid2);
      const float d0 = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(fmaxf(c2.x, 0.f))));
      const float d1 = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(fmaxf(c2.y, 0.f))));
      e = __ffma2_rn(P.q1, make_float2(d0 * d0, d1 * d1), lw);
      sf = make_float2(sinc_pi(d0 * P.inv_a), sinc_pi(d1 * P.inv_a));
    } else if (BIG) {
      const float2 c2 = __fadd2_rn(x, P.mid2);
      const float d0 = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(c2.x)));
      const float d1 = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(c2.y)));
      const float2 d2 = make_float2(d0 * d0, d1 * d1);
      if (KT == CG_GAUSS1D) {
        e = __ffma2_rn(P.q1, d2, lw);
      } else {
        const float2 ap = __ffma2_rn(dx, T.f1x, __ffma2_rn(dy, T.f1y, __fmul2_rn(dz, T.f1z)));
        const float2 bp = __ffma2_rn(dx, T.f2x, __ffma2_rn(dy, T.f2y, __fmul2_rn(dz, T.f2z)));
        const float2 s2 = __ffma2_rn(ap, ap, __fmul2_rn(bp, bp));
        const float2 ratio = make_float2((s2.x > 0.f) ? __fdividef(d2.x, s2.x) : 1.f,
                                         (s2.y > 0.f) ? __fdividef(d2.y, s2.y) : 1.f);
        const float2 t = __ffma2_rn(__fmul2_rn(P.q1, ap), ap, __fmul2_rn(__fmul2_rn(P.q4, bp), bp));
        e = __ffma2_rn(t, ratio, lw);
      }
    } else if (KT == CG_GAUSS1D) {
      e = __ffma2_rn(x, __ffma2_rn(x, P.q2, P.q1x), lw);
    } else {
      // (d / sin d)^2 = 1 + c^2/3 + 17 c^4/180 (+ O(c^6))
      const float2 c2 = __fadd2_rn(x, P.mid2);
      const float2 ap = __ffma2_rn(dx, T.f1x, __ffma2_rn(dy, T.f1y, __fmul2_rn(dz, T.f1z)));
      const float2 bp = __ffma2_rn(dx, T.f2x, __ffma2_rn(dy, T.f2y, __fmul2_rn(dz, T.f2z)));
      const float2 ratio = __ffma2_rn(c2, __ffma2_rn(c2, make_float2(17.f / 180.f, 17.f / 180.f),
                                                     make_float2(1.f / 3.f, 1.f / 3.f)),
                                      make_float2(1.f, 1.f));
      const float2 t = __ffma2_rn(__fmul2_rn(P.q1, ap), ap, __fmul2_rn(__fmul2_rn(P.q4, bp), bp));
      e = __ffma2_rn(t, ratio, lw);
    }
    const bool in0 = x.x <= P.hw, in1 = x.y <= P.hw;
    w[2 * j] = in0 ? ex2_approx(e.x) * sf.x : 0.f;
    w[2 * j + 1] = in1 ? ex2_approx(e.y) * sf.y : 0.f;
    np += (in0 ? 1u : 0u) + (in1 ? 1u : 0u);
    bm = fminf(bm, fminf(fabsf(x.x), fabsf(x.y)));
  }
  // rare: pairs inside the guard band are decided from the FP64 coordinates
  if (bm <= P.hw) {
    const uint32_t kill = band_fixup(cand, cidx, N, T, P.nmid.x, P.hw, a.tll, a.sll, slot, a.kd);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (kill & (1u << k)) {
        w[k] = 0.f;
        --np;
      }
  }
}

template <int KT, bool SPLIT, bool BIG>
__global__ void __launch_bounds__(kThreads, 1) k_grid_tc(const __grid_constant__ CUtensorMap tmap,
                                                         TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr int ns = kNS;
  const int cp = a.cp;
  Smem S;
  {
    uint8_t* p = smem_raw;
    S.B = p;
    p += (size_t)ns * cp * 64;
    S.cand = reinterpret_cast<float*>(p);
    p += (size_t)ns * kK * 4 * sizeof(float);
    S.reach = reinterpret_cast<float*>(p);
    p += (size_t)ns * 4 * kK * sizeof(float);
    S.cidx = reinterpret_cast<uint32_t*>(p);
    p += (size_t)ns * kK * sizeof(uint32_t);
    S.wpart = reinterpret_cast<float2*>(p);
    p += (size_t)2 * (kWW / 4) * kT * sizeof(float2);
    S.epi = reinterpret_cast<float*>(p);
    p += (size_t)kEW * 32 * kEpiPitch * sizeof(float);
    S.full = reinterpret_cast<uint64_t*>(p);
    S.cfull = S.full + kMaxStages;
    S.afull = S.cfull + kMaxStages;
    S.empty = S.afull + kMaxStages;
    S.dfull = S.empty + kMaxStages;
    S.dempty = S.dfull + 1;
    S.fin = S.dempty + 1;
    S.wfull = S.fin + 1;
    S.wempty = S.wfull + 2;
    S.tmem_base = reinterpret_cast<uint32_t*>(S.wempty + 2);
    S.abort_flag = reinterpret_cast<int*>(S.tmem_base + 1);
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(S.tmem_base)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&S.full[s], 1);          // producer lane 0 (+ TMA transaction bytes)
      mbar_init(&S.cfull[s], 32);        // producer lanes, after their vector stores
      mbar_init(&S.afull[s], kWW * 32);  // every weight thread
      mbar_init(&S.empty[s], 1);         // MMA commit
    }
    mbar_init(S.dfull, 1);
    mbar_init(S.dempty, kEW * 32);
    mbar_init(S.fin, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.wfull[b], kWW * 32);
      mbar_init(&S.wempty[b], kEW * 32);
    }
    *S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *S.tmem_base;
  const uint32_t tmem_d = tmem;              // columns [0, cp)
  const uint32_t acols = SPLIT ? 32u : 16u;     // TMEM columns of A per stage
  const uint32_t tmem_a = tmem + (uint32_t)cp;  // columns [cp, cp + acols ns)
  const int64_t n_items = a.n_tiles * a.n_slabs;
  volatile int* abort_flag = S.abort_flag;

  if (warp >= kProdWarp && warp < kProdWarp + kNP) {
    // ------------------------------------------------------------ producers
    const int pw = warp - kProdWarp;
    if (a.hold) {
      // testing hook: wait for a word that nothing sets; the wait runs out
      // and the kernel takes its time-out path (no copies issued yet)
      const long long t0 = clock64();
      while (*((volatile const int*)a.hold) == 0 && !*S.abort_flag &&
             clock64() - t0 < a.hold_cycles)
        __nanosleep(1000);
      if (*((volatile const int*)a.hold) == 0) {
        set_error(a.err, ERR_TIMEOUT);
        *S.abort_flag = 1;
      }
    }
    const float e_mid = make_pair_const<KT, BIG>(a.kd).e_mid;
    const int nblk = cp / 64;                     // 64-channel blocks of a slab
    const uint32_t bytes = (uint32_t)kK * (uint32_t)cp * 2u;
    int64_t k = 0;
    int64_t item = item_at(a, n_items, 0);
    int ch = 0;
    int nch = (item >= 0) ? chunks_of(a, item) : 0;
    advance(a, n_items, k, item, ch, nch, pw);
    uint32_t q = (uint32_t)pw;
    Fetch f;
    if (item >= 0) fetch_chunk(a, item, ch, lane, f);
    while (item >= 0 && !*abort_flag) {
      const int st = (int)(q % (uint32_t)kNS);
      if (q >= (uint32_t)kNS &&
          !mbar_wait(&S.empty[st], ((q / kNS) - 1) & 1, abort_flag)) {
        set_error(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      // candidate vectors: padding lies far from every target and from the
      // empty-slot sentinel (4, 4, 4) of the tile-relative target vectors
      float4 cb = make_float4(-4.f, -4.f, -4.f, -INFINITY);
      if (f.pos >= 0) {
        const float w = f.h.w;
        cb = make_float4(df_diff(f.h.x, f.l.x, f.chi.x, f.clo.x),
                         df_diff(f.h.y, f.l.y, f.chi.y, f.clo.y),
                         df_diff(f.h.z, f.l.z, f.chi.z, f.clo.z),
                         (w > 0.f) ? log2f(w) : -INFINITY);
      }
      {
        // pair-major: candidates 2j, 2j + 1 share the block j of 8 floats
        float* blk = S.cand + (size_t)st * kK * 4 + 8 * (lane >> 1) + (lane & 1);
        blk[0] = cb.x;
        blk[2] = cb.y;
        blk[4] = cb.z;
        blk[6] = cb.w + e_mid;
      }
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const float ex = cb.x - f.sq[qq].x, ey = cb.y - f.sq[qq].y, ez = cb.z - f.sq[qq].z;
        S.reach[(st * 4 + qq) * kK + lane] = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      }
      S.cidx[st * kK + lane] = f.idx;
      mbar_arrive(&S.cfull[st]);
      // data rows -> B stage: lane (j, h) gathers rows 4h .. 4h + 3 of
      // channel block j (SW128: 8-row atoms 1 KB apart, 4-row halves 512 B)
      {
        const uint32_t bbase = su32(S.B + (size_t)st * cp * 64);
        int rowk[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t rid = __shfl_sync(0xffffffffu, f.idx, (lane & 7) * 4 + t);
          rowk[t] = (rid == 0xffffffffu) ? a.n_rows : (int)rid;   // past the end: zeros
        }
        if (lane == 0)
          asm volatile(
              "{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                  su32(&S.full[st])),
              "r"(bytes)
              : "memory");
        __syncwarp();
        if (lane < nblk * 8) {
          const int j = lane >> 3, h = lane & 7;
          const uint32_t dst = bbase + (uint32_t)j * 4096u + (uint32_t)(h >> 1) * 1024u +
                               (uint32_t)(h & 1) * 512u;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(f.c_base + 64 * j), "r"(rowk[0]),
              "r"(rowk[1]), "r"(rowk[2]), "r"(rowk[3]), "r"(su32(&S.full[st]))
              : "memory");
        }
      }
      // next own chunk: issue its loads now, consume them after the next wait
      advance(a, n_items, k, item, ch, nch, kNP);
      q += kNP;
      if (item >= 0) fetch_chunk(a, item, ch, lane, f);
    }
  } else if (warp >= kEpiWarp && warp < kEpiWarp + kEW) {
    // ------------------------------------------------------------ epilogue
    // W from the weight warps' partials; once the item's MMAs are complete,
    // D (this quarter's 32 TMEM lanes, all slab columns) is normalised and
    // written; then D is released to the next item's MMAs.
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    constexpr int kGroups = kWW / 4;
    uint32_t tq = 0;
    for (int64_t item = item_at(a, n_items, 0); item >= 0 && !*abort_flag;
         item = item_at(a, n_items, (int64_t)tq + 1), ++tq) {
      const int64_t tile = item / a.n_slabs;
      const int slab = (int)(item % a.n_slabs);
      const int c_base = slab * cp;
      const int64_t slot = tile * kT + row;
      const uint32_t user = a.perm_t[slot];
      const int nch = chunks_of(a, item);
      const int wb = (int)(tq & 1);
      if (!mbar_wait(&S.wfull[wb], (tq >> 1) & 1, abort_flag)) {
        set_error(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      float W = 0.f;
#pragma unroll
      for (int g2 = 0; g2 < kGroups; ++g2) {
        const float2 o = S.wpart[((size_t)wb * kGroups + g2) * kT + row];
        W += o.x + o.y;
      }
      mbar_arrive(&S.wempty[wb]);
      if (!mbar_wait(S.dfull, tq & 1, abort_flag)) {
        set_error(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      fence_after();
      bool valid = user != 0xffffffffu;
      if (valid && (int64_t)user >= a.P) {  // never expected: record and skip
        set_error(a.err, ERR_INTERNAL);
        valid = false;
      }
      const float invW = (W > 0.f) ? 1.f / W : __int_as_float(0x7fc00000);
      // A non-finite channel value of one candidate reaches every row of the
      // MMA (0 x NaN, w x Inf): its column is non-finite in all 128 rows.
      // Flagged rows are computed again by the fix-up pass (paper Eq. 1-2:
      // only the pairs inside the support take part).  A sum of a row's
      // values turns non-finite when one of them is (or, harmlessly, on an
      // overflow, which only sends the row to the exact fix-up).
      // Accumulating calls check every row first and leave flagged rows
      // untouched; one-shot calls write the rows, and the first epilogue
      // warp's rows stand for the whole tile (every row of a contaminated
      // tile is flagged, the fix-up overwrites them).
      float2 fin2 = make_float2(0.f, 0.f);
      const bool chk_tile = a.mode == 2 && nch && warp == kEpiWarp;
      if (a.mode != 2 && nch) {
        for (int cb = 0; cb < cp; cb += 16) {
          uint32_t r[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
              "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(tmem_d + lane_off + (uint32_t)cb));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; j += 2)
            fin2 = __fadd2_rn(fin2, make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])));
        }
      }
      // accumulating call, row flagged: leave it to the fix-up
      const bool keep = !(a.mode != 2 && !isfinite(fin2.x + fin2.y));
      // one-shot output: 32 x 32 blocks through a padded shared tile so that
      // every store instruction writes 4 whole 128-byte rows
      const bool fast = a.mode == 2 && (a.C & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
      float* tile_s = S.epi + (size_t)(warp - kEpiWarp) * 32 * kEpiPitch;
      for (int cb = 0; cb < cp; cb += 32) {
        const int c0 = c_base + cb;
        // both 16-column loads in flight before one wait
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem_d + lane_off + (uint32_t)cb));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tmem_d + lane_off + (uint32_t)(cb + 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (chk_tile) {
#pragma unroll
          for (int j = 0; j < 32; j += 2)
            fin2 = __fadd2_rn(fin2, make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c1 = c0 + 16 * h;
          if (fast) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              *reinterpret_cast<float4*>(tile_s + lane * kEpiPitch + 16 * h + j) =
                  make_float4(nch ? __uint_as_float(r[16 * h + j]) * invW : invW,
                              nch ? __uint_as_float(r[16 * h + j + 1]) * invW : invW,
                              nch ? __uint_as_float(r[16 * h + j + 2]) * invW : invW,
                              nch ? __uint_as_float(r[16 * h + j + 3]) * invW : invW);
          } else if (valid && a.mode == 2) {
            float* dst = a.out + (size_t)user * a.C + c1;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c1 + j < a.C) dst[j] = nch ? __uint_as_float(r[16 * h + j]) * invW : invW;
          } else if (valid && keep) {
            float* dst = a.acc_num + (size_t)slot * a.C + c1;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (c1 + j >= a.C) continue;
              const float v = nch ? __uint_as_float(r[16 * h + j]) : 0.f;
              dst[j] = (a.mode == 1) ? dst[j] + v : v;
            }
          }
        }
        if (!fast) continue;
        __syncwarp();
        // lane: row 4 k + lane / 8 of the block, columns 4 (lane % 8) .. + 3
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int rr = 4 * k + (lane >> 3);
          const int cc = 4 * (lane & 7);
          const uint32_t u = __shfl_sync(0xffffffffu, valid ? user : 0xffffffffu, rr);
          const float4 v = *reinterpret_cast<const float4*>(tile_s + rr * kEpiPitch + cc);
          if (u != 0xffffffffu && c0 + cc < a.C)
            *reinterpret_cast<float4*>(a.out + (size_t)u * a.C + c0 + cc) = v;
        }
        __syncwarp();
      }
      if (chk_tile) {
        if (__any_sync(0xffffffffu, !isfinite(fin2.x + fin2.y))) {
#pragma unroll
          for (int q2 = 0; q2 < kT / 32; ++q2) {
            const uint64_t e = (uint64_t)(tile * kT + 32 * q2 + lane) * (uint64_t)a.n_slabs + (uint64_t)slab;
            atomicOr(&a.nf_bits[e >> 5], 1u << (e & 31));
          }
          if (lane == 0) atomicOr(a.nf_any, 1u);
        }
      } else if (a.mode != 2 && valid && nch && !isfinite(fin2.x + fin2.y)) {
        const uint64_t e = (uint64_t)slot * (uint64_t)a.n_slabs + (uint64_t)slab;
        atomicOr(&a.nf_bits[e >> 5], 1u << (e & 31));
        atomicOr(a.nf_any, 1u);
      }
      if (valid && slab == 0) {
        if (a.mode == 2) {
          if (a.out_w) a.out_w[user] = W;
        } else {
          float2 old = (a.mode == 1) ? a.acc_w[slot] : make_float2(0.f, 0.f);
          const float t = old.x + W;
          const float bp = t - old.x;
          const float err = (old.x - (t - bp)) + (W - bp);
          a.acc_w[slot] = make_float2(t, old.y + err);
        }
      }
      fence_before();
      mbar_arrive(S.dempty);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      uint32_t q = 0, tq = 0;
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) |
                             ((uint32_t)(cp >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);
      for (int64_t item = item_at(a, n_items, 0); item >= 0 && !*abort_flag;
           item = item_at(a, n_items, (int64_t)tq + 1), ++tq) {
        const int nch = chunks_of(a, item);
        if (tq > 0 && !mbar_wait(S.dempty, (tq - 1) & 1, abort_flag)) {
          set_error(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
          break;
        }
        fence_after();
        bool ok = true;
        for (int ch = 0; ch < nch; ++ch, ++q) {
          const int st = (int)(q % (uint32_t)kNS);
          const uint32_t ph = (q / kNS) & 1;
          if (!mbar_wait(&S.full[st], ph, abort_flag) ||
              !mbar_wait(&S.afull[st], ph, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t bstage = su32(S.B + (size_t)st * cp * 64);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            // SW128 MN-major: 8-candidate groups 1 KB apart, 64-channel blocks 4 KB apart
            const uint64_t bd = smem_desc_sw128(bstage + kk * 2048u, 4096u, 1024u);
#pragma unroll
            for (int h = 0; h < (SPLIT ? 2 : 1); ++h) {
              // A of candidates 16 kk .. 16 kk + 15: hi at +0, lo at +8 columns
              const uint32_t at = tmem_a + st * acols + (uint32_t)(kk * (SPLIT ? 16 : 8) + h * 8);
              const uint32_t acc = (ch > 0 || kk > 0 || h > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
                  "r"(at), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
            }
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  su32(&S.empty[st]))
              : "memory");
        }
        if (!ok) {
          set_error(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
          break;
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(S.dfull))
            : "memory");
      }
      // completion of everything this thread issued, before TMEM is freed
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(S.fin))
          : "memory");
    }
  } else {
    // ------------------------------------------------------------ weights
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;      // TMEM lane = target row
    const int grp = warp >> 2;                // candidates 16 grp .. 16 grp + 15
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const float rc = sqrtf(a.kd.c2_out);      // support radius as a chord
    const PairConst P = make_pair_const<KT, BIG>(a.kd);
    uint32_t q = 0, tq = 0;
    unsigned npair = 0;
    for (int64_t item = item_at(a, n_items, 0); item >= 0 && !*abort_flag;
         item = item_at(a, n_items, (int64_t)tq + 1), ++tq) {
      const int64_t tile = item / a.n_slabs;
      const int slab = (int)(item % a.n_slabs);
      const int64_t slot = tile * kT + row;
      if (slot >= a.n_slots) set_error(a.err, ERR_INTERNAL);
      TgtConst T;
      {
        const float4 at = a.ta[slot];
        T.nx = make_float2(-at.x, -at.x);
        T.ny = make_float2(-at.y, -at.y);
        T.nz = make_float2(-at.z, -at.z);
        float4 f1 = make_float4(0.f, 0.f, 0.f, 0.f), f2 = f1;
        if (KT == CG_GAUSS2D) {
          f1 = a.f1[slot];
          f2 = a.f2[slot];
        }
        T.f1x = make_float2(f1.x, f1.x);
        T.f1y = make_float2(f1.y, f1.y);
        T.f1z = make_float2(f1.z, f1.z);
        T.f2x = make_float2(f2.x, f2.x);
        T.f2y = make_float2(f2.y, f2.y);
        T.f2z = make_float2(f2.z, f2.z);
      }
      const int nch = chunks_of(a, item);
      // the quarter's reach: candidates beyond (quarter radius + r) give w = 0
      const float4 sq = a.subf[tile * 4 + quarter];
      const float reach2 = (rc + sq.w) * (rc + sq.w) * 1.0001f + 1e-12f;
      float ws = 0.f, wc = 0.f;
      unsigned np_item = 0;
      bool ok = true;
      for (int ch = 0; ch < nch; ++ch, ++q) {
        const int st = (int)(q % (uint32_t)kNS);
        if (!mbar_wait(&S.cfull[st], (q / kNS) & 1, abort_flag)) {
          ok = false;
          break;
        }
        // ---- 2 x 8 weights of this thread's row, branch-free ----
        // lanes 0-15 test one candidate each against the quarter's reach;
        // a group of 8 with none in reach is skipped
        const int kb = st * kK + grp * 16;
        bool reach = false;
        if (lane < 16) reach = S.reach[(st * 4 + quarter) * kK + grp * 16 + lane] <= reach2;
        const uint32_t live = __ballot_sync(0xffffffffu, reach);
        float w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = 0.f;
        const float* cg = S.cand + (size_t)kb * 4;
        if (live & 0xffu)
          eval_group<8, KT, BIG>(cg, S.cidx + kb, T, P, a, slot, w, np_item);
        if (live & 0xff00u)
          eval_group<8, KT, BIG>(cg + 32, S.cidx + kb + 8, T, P, a, slot, w + 8, np_item);
        uint32_t packed[8], packed_lo[8];
        float2 part2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2 wp = make_float2(w[2 * j], w[2 * j + 1]);
          part2 = __fadd2_rn(part2, wp);
          if (SPLIT) {
            // w = w_hi + w_lo: w_hi keeps the top 8 significand bits (exact
            // truncation), w_lo = w - w_hi is exact in FP32, then rounded
            const uint32_t u0 = __float_as_uint(wp.x), u1 = __float_as_uint(wp.y);
            packed[j] = __byte_perm(u0, u1, 0x7632);
            const float2 hi = make_float2(__uint_as_float(u0 & 0xffff0000u),
                                          __uint_as_float(u1 & 0xffff0000u));
            const float2 lo = __ffma2_rn(hi, make_float2(-1.f, -1.f), wp);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(lo.x, lo.y);
            packed_lo[j] = *reinterpret_cast<const uint32_t*>(&l2);
          } else {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(w[2 * j], w[2 * j + 1]);
            packed[j] = *reinterpret_cast<const uint32_t*>(&b2);
            packed_lo[j] = 0u;
          }
        }
        // Kahan accumulation of the chunk partial into the weight map
        {
          const float y = (part2.x + part2.y) - wc;
          const float t = ws + y;
          wc = (t - ws) - y;
          ws = t;
        }
        {
          // candidates 16 grp .. 16 grp + 15 = K step grp: split: hi at
          // columns 16 grp .. + 7, lo at 16 grp + 8 .. + 15; single: 8 grp
          const uint32_t col = SPLIT ? (uint32_t)(grp * 16) : (uint32_t)(grp * 8);
          const uint32_t ta_addr = tmem_a + lane_off + st * acols + col;
          asm volatile(
              "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                  ta_addr),
              "r"(packed[0]), "r"(packed[1]), "r"(packed[2]), "r"(packed[3]), "r"(packed[4]),
              "r"(packed[5]), "r"(packed[6]), "r"(packed[7])
              : "memory");
          if (SPLIT)
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                    ta_addr + 8u),
                "r"(packed_lo[0]), "r"(packed_lo[1]), "r"(packed_lo[2]), "r"(packed_lo[3]),
                "r"(packed_lo[4]), "r"(packed_lo[5]), "r"(packed_lo[6]), "r"(packed_lo[7])
                : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
        mbar_arrive(&S.afull[st]);
      }
      if (slab == 0) npair += np_item;
      // ---- hand this row's weight-map partial to the epilogue warps ----
      constexpr int kGroups = kWW / 4;
      const int wb = (int)(tq & 1);
      if (ok && tq >= 2 && !mbar_wait(&S.wempty[wb], ((tq >> 1) - 1) & 1, abort_flag)) ok = false;
      if (!ok) {
        set_error(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      S.wpart[((size_t)wb * kGroups + grp) * kT + row] = make_float2(ws, wc);
      mbar_arrive(&S.wfull[wb]);
    }
    unsigned c = npair;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c) atomicAdd(a.pairs, (unsigned long long)c);
  }

  // ---- teardown: all MMAs done before TMEM is released ----
  fence_before();
  __syncthreads();
  if (warp == 0) {
    int no_abort = 0;
    if (!mbar_wait(S.fin, 0, &no_abort)) set_error(a.err, ERR_TIMEOUT);
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}

// The persistent schedule (item_at): items in tile order -- the k-d order of
// the targets, so consecutive items are neighbours on the sky -- cut into
// waves of G, one item per CTA.  Inside a wave the items are ranked by cost
// (the tile's chunks + 8, the epilogue's share of an item) and the ranks
// dealt to the CTAs forwards on even waves and backwards on odd ones, so
// that the CTAs' totals stay close while the items running at any time stay
// within a wave or two: a compact patch of sky whose candidate rows the
// 129 MB L2 can hold, instead of a cost-ranked scatter of tiles that each
// read their halo from DRAM.  One CTA per wave; a bitonic sort of the wave's
// (cost, item) keys; CTAs left without an item in the last wave get -1.
// The assignment changes no result (every item is computed whole by one CTA).
constexpr int kWaveThreads = 512;
constexpr int kWaveMax = 1024;   // G <= kWaveMax

__global__ void __launch_bounds__(kWaveThreads) k_item_waves(const int32_t* __restrict__ tile_cand,
                                                             int n_slabs, int64_t n_items, int G,
                                                             int32_t* __restrict__ order) {
  __shared__ uint64_t key[kWaveMax];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * G;
  const int64_t left = n_items - base;
  const int n = left < (int64_t)G ? (int)left : G;
  int P = 1;
  while (P < G) P <<= 1;
  for (int i = tid; i < P; i += kWaveThreads) {
    uint64_t k = 0;   // padding sorts last
    if (i < n) {
      const int64_t it = base + i;
      const uint32_t cost = (uint32_t)((tile_cand[it / n_slabs] + kK - 1) / kK + 8);
      // descending cost, then ascending item (the key holds ~item)
      k = ((uint64_t)cost << 32) | (uint64_t)(0xffffffffu - (uint32_t)it);
    }
    key[i] = k;
  }
  __syncthreads();
  // bitonic sort, descending
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int i = tid; i < P; i += kWaveThreads) {
        const int l = i ^ jj;
        if (l > i) {
          const uint64_t x = key[i], y = key[l];
          const bool desc = (i & kk) == 0;
          if (desc ? (x < y) : (x > y)) {
            key[i] = y;
            key[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int r = tid; r < G; r += kWaveThreads) {
    const int cta = (blockIdx.x & 1) ? G - 1 - r : r;
    order[base + cta] =
        r < n ? (int32_t)(0xffffffffu - (uint32_t)(key[r] & 0xffffffffu)) : -1;
  }
}

using KernFn = void (*)(const CUtensorMap, TcArgs);
KernFn pick_kernel(int kt, bool split, bool big) {
  if (kt == CG_TSINC)
    return split ? k_grid_tc<CG_TSINC, true, true> : k_grid_tc<CG_TSINC, false, true>;
  if (kt == CG_GAUSS1D) {
    if (big) return split ? k_grid_tc<CG_GAUSS1D, true, true> : k_grid_tc<CG_GAUSS1D, false, true>;
    return split ? k_grid_tc<CG_GAUSS1D, true, false> : k_grid_tc<CG_GAUSS1D, false, false>;
  }
  if (big) return split ? k_grid_tc<CG_GAUSS2D, true, true> : k_grid_tc<CG_GAUSS2D, false, true>;
  return split ? k_grid_tc<CG_GAUSS2D, true, false> : k_grid_tc<CG_GAUSS2D, false, false>;
}

size_t smem_bytes(int cp, int ns) {
  return (size_t)ns * cp * 64 + (size_t)ns * kK * (sizeof(float4) + 4 * sizeof(float) + sizeof(uint32_t)) +
         (size_t)2 * (kWW / 4) * kT * sizeof(float2) + (size_t)kEW * 32 * kEpiPitch * 4 +
         (4 * kMaxStages + 7) * sizeof(uint64_t) +
         16;
}

}  // namespace

bool tc_supported(const cg_grid* g, int dtype, const void* data) {
  return dtype == CG_BF16 && g->C % 8 == 0 && (reinterpret_cast<uintptr_t>(data) % 16) == 0;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

cudaError_t grid_tiles_tc(cg_grid* g, const void* data, int mode, float* out, float* out_w, int split) {
  const Tiling& t = g->t128;
  TcArgs a;
  a.chi = t.chi;
  a.clo = t.clo;
  a.ta = t.a;
  a.subf = t.subf;
  a.range_off = t.range_off;
  a.range_s = t.range_s;
  a.range_c = t.range_c;
  a.tile_cand = t.tile_cand;
  a.n_tiles = t.n_tiles;
  a.f1 = g->tgt_f1;
  a.f2 = g->tgt_f2;
  a.tll = g->tgt_ll;
  a.perm_t = g->tgt_perm;
  a.s_hi = g->s_hi;
  a.s_lo = g->s_lo;
  a.sperm = g->sorted_val;
  a.sll = g->s_ll;
  a.data = static_cast<const __nv_bfloat16*>(data);
  a.C = g->C;
  const int slab = g->C < 256 ? g->C : 256;
  a.cp = (slab + 63) / 64 * 64;
  a.n_slabs = (g->C + a.cp - 1) / a.cp;
  a.kd = g->kdev;
  a.mode = mode;
  a.acc_num = g->acc_num;
  a.acc_w = g->acc_w;
  a.out = out;
  a.out_w = out_w;
  a.n_rows = (int)g->last_n;
  a.P = g->P;
  a.n_slots = g->n_slots;
  a.pairs = g->d_pairs;
  a.err = g->d_err;
  {
    cudaError_t ea = nonfinite_prepare(g, g->n_slots * (int64_t)a.n_slabs);
    if (ea != cudaSuccess) return ea;
    a.nf_bits = g->nf_bits;
    a.nf_any = g->nf_any;
  }
  a.hold = (g->hold && g->d_hold) ? g->d_hold : nullptr;
  a.hold_cycles = g->hold_cycles;
  // Stages: chunk q uses stage q % ns and is staged by producer warp q % kNP.
  // ns must be a multiple of kNP so that every stage always belongs to the
  // same producer warp: the parity-based empty-barrier wait is only valid
  // while its waiter is at most one phase ahead, and two producers sharing a
  // stage would also interleave their transaction counts on its barrier.
  // 8 stages of split weights (32 TMEM columns each) plus a 256-column
  // accumulator fill 512 columns.
  a.split = split ? 1 : 0;
  constexpr int ns = kNS;
  static_assert(kNS % kNP == 0, "stages must be a multiple of the producer warps");
  const uint32_t acols = split ? 32u : 16u;
  uint32_t need = (uint32_t)a.cp + acols * ns;
  uint32_t cols = 32;
  while (cols < need) cols <<= 1;
  a.tmem_cols = cols;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = smem_bytes(a.cp, ns);
  // a CTA holding 512 TMEM columns must be alone on its SM: request enough
  // shared memory that a second CTA cannot become resident
  const int per_sm = (cols > 256) ? 1 : 2;
  if (per_sm == 1 && smem < 120 * 1024) smem = 120 * 1024;
  const int64_t items = a.n_tiles * a.n_slabs;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > items) grid = items;
  if (grid < 1) return cudaSuccess;
  // balanced persistent schedule with several items per CTA: waves of
  // neighbouring items, ranked by cost inside each wave (k_item_waves)
  a.order = nullptr;
  if (items > grid && items <= INT32_MAX && grid <= kWaveMax) {
    Tiling& tw = g->t128;
    const int64_t waves = (items + grid - 1) / grid;
    if (tw.cap_order < waves * grid) {
      dfree(tw.order, g->stream);
      tw.cap_order = 0;
      cudaError_t ea = dalloc(&tw.order, (size_t)(waves * grid), g->stream);
      if (ea != cudaSuccess) return ea;
      tw.cap_order = waves * grid;
    }
    k_item_waves<<<(unsigned)waves, kWaveThreads, 0, g->stream>>>(t.tile_cand, a.n_slabs, items,
                                                                  (int)grid, tw.order);
    g->n_launches += 1;
    a.order = tw.order;
  }
  // tensor map over the caller's [N][C] BF16 rows: 64-channel x 1-row boxes,
  // 128-byte swizzle (the layout of the MMA's B operand); rows past N read 0
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)g->C, (cuuint64_t)g->last_n};
  const cuuint64_t gstride[1] = {(cuuint64_t)g->C * 2};
  const cuuint32_t box[2] = {64, 1};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(data), gdim, gstride, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // the series form drops the c^4/90 term of d^2, which changes the exponent
  // by |k1| c2^3 / 90; where that could exceed 1e-9 at the support radius the
  // exact 2 asin(c / 2) form is used instead
  const double c2o = g->kdev.c2_out;
  const bool big = g->kdev.big_support != 0 || std::fabs(g->kdev.k1) * c2o * c2o * c2o / 90.0 > 1e-9;
  auto kern = pick_kernel(a.kd.type, split != 0, big);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kThreads, smem, g->stream>>>(tmap, a);
  g->n_launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  NonfiniteRows rows;
  rows.tiling = &g->t128;
  rows.data = data;
  rows.dtype = CG_BF16;
  rows.C = g->C;
  rows.cp = a.cp;
  rows.n_slabs = a.n_slabs;
  rows.mode = mode;
  rows.out = out;
  rows.acc_num = g->acc_num;
  rows.kd = g->kdev;
  return nonfinite_fixup(g, rows);
}

}  // namespace cg
