// k_healpix.cu -- the HEALPix lookup of the paper (Sect. 2.2, 3.3, 3.4) on
// the GPU, reorganised around target tiles instead of per-sample discs:
//
//   samples:  RING index of every sample (Sect. 2.2 step 3a), a stable sort by
//             index (replacing the hash tables of Sect. 3.4), per-ring offsets
//             into the sorted order, and the sorted samples' unit vectors;
//   tiles:    one disc query per tile of targets (Sect. 2.2 step 3b, done once
//             per tile rather than once per sample), radius = tile radius +
//             support, as closed-form pixel intervals per ring (the per-ring
//             treatment of Sect. 3.3);
//   ranges:   each pixel interval becomes a contiguous range of sorted samples
//             by two binary searches inside its ring.
#include "cg_common.cuh"
#include "cg_internal.h"
#include "cg_trig.cuh"
#include "cg_healpix.cuh"

namespace cg {
namespace {

// One warp per tile; mode 0 counts ranges, mode 1 writes them.  The tile's
// candidates are the samples within r of any of its 4-target groups' discs
// (radius group radius + r): per ring, the hull of those discs' pixel
// intervals, which follows the outline of the tile widened by r (one disc of
// radius tile radius + r around the centre would hold ~1.4x as many samples
// for a square tile).  Without groups: that one disc.
constexpr int kQueryWarps = 8;
constexpr int kMaxDiscs = 32;

__global__ void __launch_bounds__(32 * kQueryWarps) k_tile_query(
    const double4* __restrict__ tc64, const double4* __restrict__ grp64, int n_grp,
    int64_t n_tiles, int64_t ns, double r_rad, int64_t* __restrict__ counts,
    const int64_t* __restrict__ offs, Range* __restrict__ out, int mode) {
  __shared__ Disc sdisc[kQueryWarps][kMaxDiscs];
  const int64_t tile = (int64_t)blockIdx.x * kQueryWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  if (tile >= n_tiles) return;
  Disc* discs = sdisc[wq];
  int nd = 1;
  if (grp64) {
    nd = n_grp;
    if (lane < nd) {
      const double4 gc = grp64[tile * nd + lane];
      Disc d = make_disc(gc, r_rad);
      if (gc.w < 0.0) d.R = -1.0;   // empty group
      discs[lane] = d;
    }
  } else if (lane == 0) {
    discs[0] = make_disc(tc64[tile], r_rad);
  }
  __syncwarp();
  // colatitude span of all discs
  double tlo = kPi, thi = 0.0;
  for (int q = 0; q < nd; ++q) {
    if (discs[q].R < 0.0) continue;
    tlo = fmin(tlo, fmax(0.0, discs[q].tc - discs[q].R));
    thi = fmax(thi, fmin(kPi, discs[q].tc + discs[q].R));
  }
  if (thi < tlo) {  // no member at all
    if (mode == 0 && lane == 0) counts[tile] = 0;
    return;
  }
  int64_t ilo = (int64_t)floor(ring_coord(ns, cos(tlo))) - 2;
  int64_t ihi = (int64_t)ceil(ring_coord(ns, cos(thi))) + 2;
  ilo = ilo < 1 ? 1 : ilo;
  ihi = ihi > 4 * ns - 1 ? 4 * ns - 1 : ihi;
  int64_t pos = (mode == 1) ? offs[tile] : 0;
  int64_t total = 0;
  for (int64_t base = ilo; base <= ihi; base += 32) {
    const int64_t i = base + lane;
    Range rr[2];
    const int n = (i <= ihi) ? ring_ranges(ns, i, discs, nd, rr) : 0;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int sum = __shfl_sync(0xffffffffu, incl, 31);
    if (mode == 1) {
      for (int q = 0; q < n; ++q) {
        rr[q].pad = (int32_t)tile;
        out[pos + incl - n + q] = rr[q];
      }
      pos += sum;
    }
    total += sum;
  }
  if (mode == 0 && lane == 0) counts[tile] = total;
}


// RING index of a valid direction and the double-float sine / cosine of its
// latitude and longitude.  Ordinary angles (|lon| < 2048 deg) take an FP64-free
// path: the inputs are split into double-float pairs with integer operations,
// the trigonometry and the index arithmetic run in double-float, and only a
// decision within the margin of a pixel boundary, the cap/belt boundary, the
// immediate neighbourhood of a pole and the caps' quadrant boundaries go to
// the FP64 routines.
__device__ __forceinline__ int64_t key_and_sincos(int64_t ns, double lo, double la, df32& sb,
                                                  df32& cb, df32& sl, df32& cl) {
  const bool fast = df_split_ok(lo) && df_split_ok(la) &&
                    (__double_as_longlong(lo) & 0x7ff0000000000000ll) < (1034ll << 52);
  bool ok = false;
  int64_t kpix = 0;
  if (fast) {
    const df32 lon_d = df_split(lo), lat_d = df_split(la);
    df_sincos_deg_df(lat_d, sb, cb);
    df_sincos_deg_df(lon_d, sl, cl);
    kpix = ang2pix_ring_df(ns, lon_d, sb, &ok);
  } else {
    df_sincos_deg(la, sb, cb);
    df_sincos_deg(lo, sl, cl);
  }
  return ok ? kpix : ang2pix_ring_dual(ns, lo, la, sb);
}

__global__ void k_ang2pix_export(int64_t ns, const double* __restrict__ lon,
                                 const double* __restrict__ lat, int64_t n,
                                 int64_t* __restrict__ pix) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo = lon[i], la = lat[i];
  if (!valid_coord(lo, la)) {
    pix[i] = -1;
    return;
  }
  df32 sb, cb, sl, cl;
  pix[i] = key_and_sincos(ns, lo, la, sb, cb, sl, cl);
}

// Unit vectors (double-float) of n directions, as FP64 [n][3].
__global__ void k_unit_vectors(const double* __restrict__ lon, const double* __restrict__ lat,
                               int64_t n, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  df32 sb, cb, sl, cl;
  df_sincos_deg(lat[i], sb, cb);
  df_sincos_deg(lon[i], sl, cl);
  const df32 x = df_mul(cb, cl), y = df_mul(cb, sl);
  out[3 * i + 0] = (double)x.hi + (double)x.lo;
  out[3 * i + 1] = (double)y.hi + (double)y.lo;
  out[3 * i + 2] = (double)sb.hi + (double)sb.lo;
}

// Per sample (input order): RING key (invalid samples get npix and sort to
// the end), identity value for the sort, and the unit vector as (hi, lo)
// FP32 pairs with w = sample weight, one 32-byte record u[2 i], u[2 i + 1].
__global__ void k_sample_keys(int64_t ns, const double* __restrict__ lon,
                              const double* __restrict__ lat,
                              const float* __restrict__ weights, int64_t n,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                              float4* __restrict__ u, double2* __restrict__ sll, unsigned* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo = lon[i], la = lat[i];
  val[i] = (uint32_t)i;
  sll[i] = make_double2(lo, la);
  if (!valid_coord(lo, la)) {
    key[i] = (uint32_t)(12 * ns * ns);
    u[2 * i] = make_float4(4.f, 4.f, 4.f, 0.f);
    u[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    set_error(err, ERR_BAD_SAMPLE);
    return;
  }
  df32 sb, cb, sl, cl;
  key[i] = (uint32_t)key_and_sincos(ns, lo, la, sb, cb, sl, cl);
  const df32 x = df_mul(cb, cl), y = df_mul(cb, sl);
  float w = 1.f;
  if (weights) {
    w = weights[i];
    if (!(w >= 0.f) || !isfinite(w)) {
      set_error(err, ERR_BAD_SAMPLE);
      w = 0.f;
    }
  }
  u[2 * i] = make_float4(x.hi, y.hi, sb.hi, w);
  u[2 * i + 1] = make_float4(x.lo, y.lo, sb.lo, 0.f);
}


// Sorted order: gather the unit vectors, and ring_off[i] = first sorted
// position with ring >= i, i = 0 .. 4 ns (thread s writes the entries for
// the rings after its predecessor's ring up to its own).
__global__ void k_sample_gather(int64_t ns, int lg, const uint32_t* __restrict__ skey,
                                const uint32_t* __restrict__ sval,
                                const float4* __restrict__ u_hi,
                                const float4* __restrict__ u_lo, int stride, int64_t n,
                                float4* __restrict__ s_hi, float4* __restrict__ s_lo,
                                int32_t* __restrict__ ring_off) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t npix = 12 * ns * ns;
  const int64_t end = 4 * ns;
  int64_t rc = end;
  if (s < n) {
    const int64_t idx = (int64_t)sval[s] * stride;
    s_hi[s] = u_hi[idx];
    s_lo[s] = u_lo[idx];
    const int64_t k = skey[s];
    rc = (k >= npix) ? end : ring_of_key(ns, lg, k);
  }
  int64_t rp = __shfl_up_sync(0xffffffffu, rc, 1);
  if (lane == 0) {
    rp = -1;
    if (s > 0 && s - 1 < n) {
      const int64_t k = skey[s - 1];
      rp = (k >= npix) ? end : ring_of_key(ns, lg, k);
    }
  }
  if (s > n) return;
  for (int64_t i = rp + 1; i <= rc; ++i) ring_off[i] = (int32_t)s;
}


// One warp per tile: the sorted-sample interval [lo, hi) of each of the
// tile's pixel ranges (binary search inside the range's ring), the number of
// the tile's candidates before each range (cum), and the tile's total.
__global__ void k_tile_ranges(const Range* __restrict__ ranges,
                              const int64_t* __restrict__ range_off, int64_t n_tiles,
                              const int32_t* __restrict__ ring_off,
                              const uint32_t* __restrict__ skey, int2* __restrict__ out,
                              int32_t* __restrict__ cum, int32_t* __restrict__ tile_cand) {
  const int64_t tile = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= n_tiles) return;
  const int64_t r0 = range_off[tile], r1 = range_off[tile + 1];
  int32_t running = 0;
  for (int64_t b = r0; b < r1; b += 32) {
    const int64_t r = b + lane;
    int32_t lo = 0, hi = 0;
    if (r < r1) {
      const Range q = ranges[r];
      const int32_t a = ring_off[q.ring], e = ring_off[q.ring + 1];
      lo = a;
      hi = a;
      if (e > a) {
        lo = lower_bound_u32(skey, a, e, (uint32_t)q.pix_lo);
        hi = lower_bound_u32(skey, lo, e, (uint32_t)q.pix_hi + 1u);
      }
    }
    const int32_t cnt = hi - lo;
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (r < r1) {
      out[r] = make_int2(lo, hi);
      cum[r] = running + incl - cnt;
    }
    running += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) tile_cand[tile] = running;
}

__global__ void k_export(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sval,
                         int64_t n, int64_t* __restrict__ pix, int64_t* __restrict__ perm) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  pix[s] = skey[s];
  perm[s] = sval[s];
}

__global__ void k_export_ring(const int32_t* __restrict__ ro, int64_t m, int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = ro[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Fused batches: the sample index of all jobs at once.
// ---------------------------------------------------------------------------
namespace {

// Largest j with off[j] <= x (off[0] = 0, x < off[n]).
__device__ __forceinline__ int batch_job(const int64_t* __restrict__ off, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// k_sample_keys for every job: composite key (job key base + RING key at the
// job's nside), the sample's index within its job, its unit vector record
// and FP64 lon/lat at its batch position.  CTA b serves 256 samples of the
// job whose CTA range (blk: prefix of the jobs' CTA counts) holds b.
__global__ void __launch_bounds__(256) k_batch_keys(const BatchIndexJob* __restrict__ jobs,
                                                    const int64_t* __restrict__ blk, int n_jobs,
                                                    uint64_t* __restrict__ key,
                                                    uint32_t* __restrict__ val,
                                                    float4* __restrict__ u,
                                                    double2* __restrict__ sll, unsigned* err) {
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = batch_job(blk, n_jobs, blockIdx.x);
  __syncthreads();
  const int j = s_job;
  const BatchIndexJob& J = jobs[j];
  const int64_t li = (int64_t)(blockIdx.x - blk[j]) * 256 + threadIdx.x;
  if (li >= J.n) return;
  const int64_t i = J.off + li;
  const int64_t ns = J.nside;
  const double lo = J.lon[li], la = J.lat[li];
  val[i] = (uint32_t)li;
  sll[i] = make_double2(lo, la);
  if (!valid_coord(lo, la)) {
    key[i] = J.key_base + (uint64_t)(12 * ns * ns);
    u[2 * i] = make_float4(4.f, 4.f, 4.f, 0.f);
    u[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    set_error(err, ERR_BAD_SAMPLE);
    return;
  }
  df32 sb, cb, sl, cl;
  key[i] = J.key_base + (uint64_t)key_and_sincos(ns, lo, la, sb, cb, sl, cl);
  const df32 x = df_mul(cb, cl), y = df_mul(cb, sl);
  float w = 1.f;
  if (J.weights) {
    w = J.weights[li];
    if (!(w >= 0.f) || !isfinite(w)) {
      set_error(err, ERR_BAD_SAMPLE);
      w = 0.f;
    }
  }
  u[2 * i] = make_float4(x.hi, y.hi, sb.hi, w);
  u[2 * i + 1] = make_float4(x.lo, y.lo, sb.lo, 0.f);
}

// k_sample_gather for every job: each thread covers one position s = 0 .. n
// of its job's segment (CTA b serves 256 of them, blk: prefix of the jobs'
// CTA counts for n + 1 positions); ring offsets are relative to the segment,
// so that each job sees its own index as if it ran alone.
__global__ void __launch_bounds__(256) k_batch_gather(const BatchIndexJob* __restrict__ jobs,
                                                      const int64_t* __restrict__ blk, int n_jobs,
                                                      const uint64_t* __restrict__ skey64,
                                                      const uint32_t* __restrict__ sval,
                                                      const float4* __restrict__ u,
                                                      float4* __restrict__ s_hi,
                                                      float4* __restrict__ s_lo,
                                                      uint32_t* __restrict__ skey,
                                                      int32_t* __restrict__ ring_off) {
  __shared__ int s_job;
  if (threadIdx.x == 0) s_job = batch_job(blk, n_jobs, blockIdx.x);
  __syncthreads();
  const int j = s_job;
  const BatchIndexJob& J = jobs[j];
  const int64_t s = (int64_t)(blockIdx.x - blk[j]) * 256 + threadIdx.x;   // 0 .. n
  if (s > J.n) return;
  const int64_t ns = J.nside;
  const int64_t npix = 12 * ns * ns;
  const int64_t end = 4 * ns;
  int64_t rc = end;
  if (s < J.n) {
    const int64_t gs = J.off + s;
    const int64_t rec = 2 * (J.off + (int64_t)sval[gs]);
    s_hi[gs] = u[rec];
    s_lo[gs] = u[rec + 1];
    const int64_t k = (int64_t)(skey64[gs] - J.key_base);
    skey[gs] = (uint32_t)k;
    rc = (k >= npix) ? end : ring_of_key(ns, J.lg, k);
  }
  int64_t rp = -1;
  if (s > 0) {
    const int64_t k = (int64_t)(skey64[J.off + s - 1] - J.key_base);
    rp = (k >= npix) ? end : ring_of_key(ns, J.lg, k);
  }
  int32_t* ro = ring_off + J.ring_base;
  for (int64_t i = rp + 1; i <= rc; ++i) ro[i] = (int32_t)s;
}

// k_tile_ranges for the tiles of every job (one warp per tile).
__global__ void k_batch_ranges(const BatchIndexJob* __restrict__ jobs,
                               const int64_t* __restrict__ tile_off, int n_jobs, int64_t n_tiles,
                               const int32_t* __restrict__ ring_off_all,
                               const uint32_t* __restrict__ skey_all) {
  const int64_t gt = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gt >= n_tiles) return;
  const int j = batch_job(tile_off, n_jobs, gt);
  const BatchIndexJob& J = jobs[j];
  const int64_t tile = gt - tile_off[j];
  const int32_t* ring_off = ring_off_all + J.ring_base;
  const uint32_t* skey = skey_all + J.off;
  const int64_t r0 = J.range_off[tile], r1 = J.range_off[tile + 1];
  int32_t running = 0;
  for (int64_t b = r0; b < r1; b += 32) {
    const int64_t r = b + lane;
    int32_t lo = 0, hi = 0;
    if (r < r1) {
      const Range q = J.ranges[r];
      const int32_t a = ring_off[q.ring], e = ring_off[q.ring + 1];
      lo = a;
      hi = a;
      if (e > a) {
        lo = lower_bound_u32(skey, a, e, (uint32_t)q.pix_lo);
        hi = lower_bound_u32(skey, lo, e, (uint32_t)q.pix_hi + 1u);
      }
    }
    const int32_t cnt = hi - lo;
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (r < r1) {
      J.range_s[r] = make_int2(lo, hi);
      J.range_c[r] = running + incl - cnt;
    }
    running += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) J.tile_cand[tile] = running;
}

}  // namespace

cudaError_t batch_index_alloc(BatchIndex& bi, cudaStream_t s) {
  const size_t n = (size_t)bi.N;
  cudaError_t e;
  if ((e = dalloc(&bi.key, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.val, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.u_rec, 2 * n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.sll, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.s_hi, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.s_lo, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.skey, n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&bi.ring_off, (size_t)bi.n_ring, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

void batch_index_free(BatchIndex& bi, cudaStream_t s) {
  dfree(bi.jobs, s);
  dfree(bi.key_blk, s);
  dfree(bi.gth_blk, s);
  dfree(bi.tile_off, s);
  dfree(bi.key, s);
  dfree(bi.val, s);
  dfree(bi.u_rec, s);
  dfree(bi.sll, s);
  dfree(bi.s_hi, s);
  dfree(bi.s_lo, s);
  dfree(bi.skey, s);
  dfree(bi.ring_off, s);
  if (bi.sw.keys_alt) cudaFreeAsync(bi.sw.keys_alt, s);
  bi.sw.keys_alt = nullptr;
  dfree(bi.sw.vals_alt, s);
  dfree(bi.sw.hist, s);
  dfree(bi.sw.totals, s);
  dfree(bi.sw.status, s);
  dfree(bi.sw.os_meta, s);
  bi.sw = SortWork();
  bi.sorted_key = nullptr;
  bi.sorted_val = nullptr;
}

cudaError_t batch_index_run(BatchIndex& bi, unsigned* err, cudaStream_t s, int64_t* launches) {
  if (bi.N <= 0) return cudaSuccess;
  k_batch_keys<<<(unsigned)bi.n_key_blk, 256, 0, s>>>(bi.jobs, bi.key_blk, bi.n_jobs, bi.key,
                                                      bi.val, bi.u_rec, bi.sll, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = radix_sort_u64(bi.key, bi.val, bi.N, bi.key_bits, bi.sw, s, &bi.sorted_key, &bi.sorted_val);
  if (e != cudaSuccess) return e;
  k_batch_gather<<<(unsigned)bi.n_gth_blk, 256, 0, s>>>(
      bi.jobs, bi.gth_blk, bi.n_jobs, bi.sorted_key, bi.sorted_val, bi.u_rec, bi.s_hi,
      bi.s_lo, bi.skey, bi.ring_off);
  if (bi.n_tiles > 0) {
    const int warps = 8;
    k_batch_ranges<<<ceil_div(bi.n_tiles, warps), 32 * warps, 0, s>>>(
        bi.jobs, bi.tile_off, bi.n_jobs, bi.n_tiles, bi.ring_off, bi.skey);
  }
  if (launches) *launches += 3 + 3 * ((bi.key_bits + 7) / 8);
  return cudaGetLastError();
}

int key_bits_for(int64_t ns) {
  const uint64_t maxkey = (uint64_t)(12 * ns * ns);  // sentinel for invalid samples
  int b = 0;
  while (b < 32 && (maxkey >> b) != 0) ++b;
  return b;
}

cudaError_t ang2pix_export(int nside, const double* lon, const double* lat, int64_t n,
                           int64_t* pix, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_ang2pix_export<<<ceil_div(n, 256), 256, 0, s>>>(nside, lon, lat, n, pix);
  return cudaGetLastError();
}

cudaError_t unit_vectors(const double* lon, const double* lat, int64_t n, double* out,
                         cudaStream_t s) {
  if (n > 0) k_unit_vectors<<<ceil_div(n, 256), 256, 0, s>>>(lon, lat, n, out);
  return cudaGetLastError();
}

void tiling_free(Tiling& t, cudaStream_t s) {
  dfree(t.chi, s);
  dfree(t.clo, s);
  dfree(t.c64, s);
  dfree(t.a, s);
  dfree(t.tile_cand, s);
  dfree(t.order, s);
  t.cap_order = 0;
  dfree(t.sub64, s);
  dfree(t.grp64, s);
  dfree(t.subf, s);
  dfree(t.range_off, s);
  dfree(t.ranges, s);
  dfree(t.range_s, s);
  dfree(t.range_c, s);
  t.n_ranges = 0;
}

cudaError_t tiles_query(cg_grid* g, Tiling& t) {
  cudaStream_t s = g->stream;
  const int64_t nt = t.n_tiles;
  const double r = g->support_deg * kDeg2Rad;
  int64_t* counts = nullptr;
  cudaError_t e;
  dfree(t.range_off, s);
  dfree(t.ranges, s);
  dfree(t.range_s, s);
  dfree(t.range_c, s);
  if ((e = dalloc(&counts, (size_t)nt, s)) != cudaSuccess) return e;
  const int n_grp = t.T / 4;
  k_tile_query<<<ceil_div(nt, kQueryWarps), 32 * kQueryWarps, 0, s>>>(
      t.c64, t.grp64, n_grp, nt, g->nside, r, counts, nullptr, nullptr, 0);
  g->n_launches += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt + 1));
  if (!h) return cudaErrorMemoryAllocation;
  e = cudaMemcpyAsync(h + 1, counts, sizeof(int64_t) * (size_t)nt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { free(h); return e; }
  h[0] = 0;
  for (int64_t i = 0; i < nt; ++i) h[i + 1] += h[i];
  t.n_ranges = h[nt];
  if ((e = dalloc(&t.range_off, (size_t)nt + 1, s)) != cudaSuccess) { free(h); return e; }
  if ((e = dalloc(&t.ranges, (size_t)t.n_ranges, s)) != cudaSuccess) { free(h); return e; }
  if ((e = dalloc(&t.range_s, (size_t)t.n_ranges, s)) != cudaSuccess) { free(h); return e; }
  if ((e = dalloc(&t.range_c, (size_t)t.n_ranges, s)) != cudaSuccess) { free(h); return e; }
  e = cudaMemcpyAsync(t.range_off, h, sizeof(int64_t) * (size_t)(nt + 1),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  free(h);
  if (e != cudaSuccess) return e;
  k_tile_query<<<ceil_div(nt, kQueryWarps), 32 * kQueryWarps, 0, s>>>(
      t.c64, t.grp64, n_grp, nt, g->nside, r, nullptr, t.range_off, t.ranges, 1);
  g->n_launches += 1;
  dfree(counts, s);
  dfree(g->ring_off, s);
  if ((e = dalloc(&g->ring_off, (size_t)(4 * g->nside + 1), s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

static cudaError_t ensure_samples(cg_grid* g, int64_t n) {
  if (g->cap_n >= (size_t)n) return cudaSuccess;
  cudaStream_t s = g->stream;
  dfree(g->key, s);
  dfree(g->val, s);
  dfree(g->s_hi, s);
  dfree(g->s_lo, s);
  dfree(g->u_rec, s);
  dfree(g->s_ll, s);
  g->cap_n = 0;
  cudaError_t e;
  if ((e = dalloc(&g->key, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->val, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->s_hi, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->s_lo, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->u_rec, 2 * (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->s_ll, (size_t)n, s)) != cudaSuccess) return e;
  g->cap_n = (size_t)n;
  return cudaSuccess;
}

cudaError_t samples_keys(cg_grid* g, const double* lon, const double* lat, const float* weights,
                         int64_t n) {
  cudaError_t e = ensure_samples(g, n);
  if (e != cudaSuccess) return e;
  k_sample_keys<<<ceil_div(n, 256), 256, 0, g->stream>>>(g->nside, lon, lat, weights, n, g->key,
                                                         g->val, g->u_rec, g->s_ll,
                                                         g->d_err);
  g->n_launches += 1;
  return cudaGetLastError();
}

cudaError_t samples_sort(cg_grid* g, int64_t n) {
  const int bits = key_bits_for(g->nside);
  g->n_launches += 1 + (bits + 7) / 8;
  g->sw.err = g->d_err;
  return radix_sort_u32(g->key, g->val, n, bits, g->sw, g->stream, &g->sorted_key,
                        &g->sorted_val);
}

cudaError_t sorted_gather(int64_t ns, const uint32_t* skey, const uint32_t* sval,
                          const float4* u_hi, const float4* u_lo, int stride, int64_t n,
                          float4* s_hi, float4* s_lo, int32_t* ring_off, cudaStream_t s) {
  int lg = -1;
  if ((ns & (ns - 1)) == 0)
    for (lg = 0; ((int64_t)1 << lg) < ns; ++lg) {
    }
  k_sample_gather<<<ceil_div(n + 1, 256), 256, 0, s>>>(ns, lg, skey, sval, u_hi, u_lo, stride, n, s_hi,
                                                       s_lo, ring_off);
  return cudaGetLastError();
}

cudaError_t samples_prepare(cg_grid* g, int64_t n) {
  cudaStream_t s = g->stream;
  const int64_t ns = g->nside;
  cudaError_t e = sorted_gather(ns, g->sorted_key, g->sorted_val, g->u_rec, g->u_rec + 1, 2, n, g->s_hi,
                                g->s_lo, g->ring_off, s);
  if (e != cudaSuccess) return e;
  g->n_launches += 1;
  g->last_n = n;
  return cudaGetLastError();
}

cudaError_t tiles_ranges(cg_grid* g, Tiling& t) {
  if (t.n_tiles > 0) {
    const int warps = 8;
    k_tile_ranges<<<ceil_div(t.n_tiles, warps), 32 * warps, 0, g->stream>>>(
        t.ranges, t.range_off, t.n_tiles, g->ring_off, g->sorted_key, t.range_s, t.range_c,
        t.tile_cand);
    g->n_launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t export_index(cg_grid* g, int64_t* sorted_pix, int64_t* perm, int64_t* ring_off,
                         int64_t n) {
  cudaStream_t s = g->stream;
  if (n > 0) k_export<<<ceil_div(n, 256), 256, 0, s>>>(g->sorted_key, g->sorted_val, n,
                                                      sorted_pix, perm);
  if (ring_off) {
    const int64_t m = 4 * (int64_t)g->nside + 1;
    k_export_ring<<<ceil_div(m, 256), 256, 0, s>>>(g->ring_off, m, ring_off);
  }
  return cudaGetLastError();
}

}  // namespace cg
