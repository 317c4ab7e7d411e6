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

namespace cg {
namespace {

struct RingGeo {
  int64_t count, first;
  double z, phase;
};

__device__ __forceinline__ RingGeo ring_geo(int64_t ns, int64_t i) {
  RingGeo r;
  const double dns = (double)ns;
  if (i < ns) {
    r.count = 4 * i;
    r.first = 2 * i * (i - 1);
    r.z = 1.0 - (double)(i * i) / (3.0 * dns * dns);
    r.phase = 0.5;
  } else if (i <= 3 * ns) {
    r.count = 4 * ns;
    r.first = 2 * ns * (ns - 1) + (i - ns) * 4 * ns;
    r.z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * dns);
    r.phase = (((i - ns) & 1) == 0) ? 0.5 : 0.0;
  } else {
    const int64_t k = 4 * ns - i;
    r.count = 4 * k;
    r.first = 12 * ns * ns - 2 * k * (k + 1);
    r.z = -(1.0 - (double)(k * k) / (3.0 * dns * dns));
    r.phase = 0.5;
  }
  return r;
}

__device__ __forceinline__ double ring_colat(int64_t ns, int64_t i) {
  if (i <= 0) return 0.0;
  if (i >= 4 * ns) return kPi;
  return acos(ring_geo(ns, i).z);
}

// Continuous ring coordinate of a direction with cos(colatitude) = z.
__device__ __forceinline__ double ring_coord(int64_t ns, double z) {
  const double dns = (double)ns;
  if (fabs(z) <= 2.0 / 3.0) return dns * (2.0 - 1.5 * z);
  if (z > 0.0) return dns * sqrt(3.0 * (1.0 - z));
  return 4.0 * dns - dns * sqrt(3.0 * (1.0 + z));
}

// Widest longitude half-width of the disc (centre colatitude tc, radius R)
// over the colatitude band [ta, tb]: -1 if the disc misses the band, >= pi if
// it covers every longitude there.  The half-width at colatitude t solves
// cos R = cos tc cos t + sin tc sin t cos(dphi); its widest point over t is
// at cos t = cos tc / cos R (or at a band edge).
__device__ double disc_halfwidth(double tc, double R, double ta, double tb) {
  if (tb < tc - R || ta > tc + R) return -1.0;
  if (ta <= 0.0 && tc <= R) return 4.0 * kPi;
  if (tb >= kPi && tc + R >= kPi) return 4.0 * kPi;
  const double st = sin(tc), ct = cos(tc), cr = cos(R);
  if (st <= 0.0) return 4.0 * kPi;
  double lo = fmax(ta, tc - R), hi = fmin(tb, tc + R);
  lo = fmax(lo, 1e-300);
  hi = fmin(hi, kPi - 1e-16);
  double ts = (fabs(ct / cr) <= 1.0) ? acos(ct / cr) : lo;
  ts = fmin(fmax(ts, lo), hi);
  double xmin = 1e300;
  const double cand[3] = {lo, hi, ts};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double x = (cr - ct * cos(cand[q])) / (st * sin(cand[q]));
    xmin = fmin(xmin, x);
  }
  if (xmin <= -1.0) return 4.0 * kPi;
  if (xmin > 1.0) return -1.0;
  return acos(xmin);
}

// A disc on the sphere: colatitude, longitude (radians) and radius.
struct Disc {
  double tc, pc, R;
};

// Pixel ranges of ring i met by the union of nd discs (the hull of their
// pixel intervals on the ring, a superset); writes up to 2 into out.
__device__ int ring_ranges(int64_t ns, int64_t i, const Disc* discs, int nd, Range* out) {
  const RingGeo g = ring_geo(ns, i);
  const double dphi = 2.0 * kPi / (double)g.count;
  const double ta = ring_colat(ns, i - 1), tb = ring_colat(ns, i + 1);
  bool any = false, full = false;
  double lo = 0.0, hi = 0.0;   // hull of [pc - W, pc + W], unwrapped near the first disc
  for (int q = 0; q < nd && !full; ++q) {
    const double hw = disc_halfwidth(discs[q].tc, discs[q].R, ta, tb);
    if (hw < 0.0) continue;
    const double W = hw + 0.5 * dphi + 1e-12;
    if (W >= kPi) { full = true; break; }
    double c = discs[q].pc;
    if (any) {  // move c to within pi of the hull's first centre
      const double ref = 0.5 * (lo + hi);
      while (c - ref > kPi) c -= 2.0 * kPi;
      while (ref - c > kPi) c += 2.0 * kPi;
      lo = fmin(lo, c - W);
      hi = fmax(hi, c + W);
    } else {
      lo = c - W;
      hi = c + W;
      any = true;
    }
  }
  if (!any && !full) return 0;
  int64_t jlo = 0, jhi = g.count - 1;
  if (!full && hi - lo >= 2.0 * kPi) full = true;
  if (!full) {
    jlo = (int64_t)ceil(lo / dphi - g.phase);
    jhi = (int64_t)floor(hi / dphi - g.phase);
    if (jhi < jlo) return 0;
    if (jhi - jlo + 1 >= g.count) full = true;
  }
  if (full) {
    if (out) out[0] = Range{(int32_t)g.first, (int32_t)(g.first + g.count - 1), (int32_t)i, 0};
    return 1;
  }
  int64_t a = jlo % g.count, b = jhi % g.count;
  if (a < 0) a += g.count;
  if (b < 0) b += g.count;
  if (a <= b) {
    if (out) out[0] = Range{(int32_t)(g.first + a), (int32_t)(g.first + b), (int32_t)i, 0};
    return 1;
  }
  if (out) {
    out[0] = Range{(int32_t)g.first, (int32_t)(g.first + b), (int32_t)i, 0};
    out[1] = Range{(int32_t)(g.first + a), (int32_t)(g.first + g.count - 1), (int32_t)i, 0};
  }
  return 2;
}

__device__ __forceinline__ Disc make_disc(double4 c, double r_rad) {
  Disc d;
  d.tc = acos(fmin(1.0, fmax(-1.0, c.z)));
  d.pc = atan2(c.y, c.x);
  d.R = c.w + r_rad;
  return d;
}

// One warp per tile; mode 0 counts ranges, mode 1 writes them.  With sub64
// the tile's candidates are those of its four quarter discs (tighter than one
// disc around the tile centre); otherwise one disc of radius (tile radius + r).
__global__ void k_tile_query(const double4* __restrict__ tc64,
                             const double4* __restrict__ sub64, int64_t n_tiles, int64_t ns,
                             double r_rad, int64_t* __restrict__ counts,
                             const int64_t* __restrict__ offs, Range* __restrict__ out,
                             int mode) {
  const int64_t tile = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= n_tiles) return;
  Disc discs[4];
  int nd = 1;
  discs[0] = make_disc(tc64[tile], r_rad);
  if (sub64) {
    nd = 4;
    for (int q = 0; q < 4; ++q) discs[q] = make_disc(sub64[tile * 4 + q], r_rad);
  }
  // colatitude span of all discs
  double tlo = kPi, thi = 0.0;
  for (int q = 0; q < nd; ++q) {
    tlo = fmin(tlo, fmax(0.0, discs[q].tc - discs[q].R));
    thi = fmax(thi, fmin(kPi, discs[q].tc + discs[q].R));
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

__device__ __forceinline__ bool valid_coord(double lon, double lat) {
  return isfinite(lon) && isfinite(lat) && lat >= -90.0 && lat <= 90.0;
}

// HEALPix RING index from an approximate z = sin(lat) (|error| ~1e-14):
// the same decisions as ang2pix_ring_f64, each checked for a margin that the
// FP64 evaluation's own rounding cannot cross; *ok = false when a value lies
// within that margin of a decision boundary (then the exact FP64 routine
// decides).  For nside <= 16384 a truncated quantity is at most 4 nside =
// 65536 and FP64 and this evaluation differ by < 1e-9 there; the margin is
// 1e-6.
__device__ __forceinline__ int64_t ang2pix_ring_fast(int64_t ns, double lon_deg, double z,
                                                     bool* ok) {
  constexpr double M = 1e-6;
  const double za = fabs(z);
  const double phi = lon_fold_deg(lon_deg);
  const double tt = phi * (1.0 / 90.0);
  const double dns = (double)ns;
  bool good = fabs(za - 2.0 / 3.0) > 1e-9;
  int64_t pix;
  if (za <= 2.0 / 3.0) {
    const double u = dns * (0.5 + tt);
    const double v = dns * (z * 0.75);
    const double A = u - v, B = u + v;
    const double fa = A - floor(A), fb = B - floor(B);
    good = good && fa > M && fa < 1.0 - M && fb > M && fb < 1.0 - M;
    const int64_t asc = (int64_t)A;
    const int64_t dsc = (int64_t)B;
    const int64_t k = ns + 1 + asc - dsc;
    const int64_t odd = k & 1;
    int64_t j = (asc + dsc - ns + (1 - odd) + 1) / 2;
    j %= 4 * ns;
    if (j < 0) j += 4 * ns;
    pix = 2 * ns * (ns - 1) + (k - 1) * 4 * ns + j;
  } else {
    const double ft = tt - floor(tt);
    // near a pole sqrt(1 - za) magnifies the error of z: leave it to FP64
    good = good && ft > 1e-12 && ft < 1.0 - 1e-12 && 1.0 - za > 1e-6;
    const double x = dns * sqrt(3.0 * (1.0 - za));
    const double P = ft * x, Q = (1.0 - ft) * x;
    const double fp = P - floor(P), fq = Q - floor(Q);
    good = good && fp > M && fp < 1.0 - M && fq > M && fq < 1.0 - M;
    const int64_t a = (int64_t)P;
    const int64_t b = (int64_t)Q;
    const int64_t k = a + b + 1;
    const double J = tt * (double)k;
    const double fj = J - floor(J);
    good = good && fj > M && fj < 1.0 - M;
    int64_t j = (int64_t)J;
    j %= 4 * k;
    if (j < 0) j += 4 * k;
    pix = (z > 0.0) ? 2 * k * (k - 1) + j : 12 * ns * ns - 2 * k * (k + 1) + j;
  }
  *ok = good;
  return pix;
}

// RING index of a valid sample with z from the double-float sine; exact
// FP64 fallback near decision boundaries.
__device__ __forceinline__ int64_t ang2pix_ring_dual(int64_t ns, double lon, double lat,
                                                     df32 sb) {
  if (ns > 16384) return ang2pix_ring_f64(ns, lon, lat);
  bool ok;
  const int64_t p = ang2pix_ring_fast(ns, lon, (double)sb.hi + (double)sb.lo, &ok);
  return ok ? p : ang2pix_ring_f64(ns, lon, lat);
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
  df32 sb, cb;
  df_sincos_deg(la, sb, cb);
  pix[i] = ang2pix_ring_dual(ns, lo, la, sb);
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
// FP32 pairs with w = sample weight.
__global__ void k_sample_keys(int64_t ns, const double* __restrict__ lon,
                              const double* __restrict__ lat,
                              const float* __restrict__ weights, int64_t n,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                              float4* __restrict__ u_hi, float4* __restrict__ u_lo,
                              unsigned* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo = lon[i], la = lat[i];
  val[i] = (uint32_t)i;
  if (!valid_coord(lo, la)) {
    key[i] = (uint32_t)(12 * ns * ns);
    u_hi[i] = make_float4(4.f, 4.f, 4.f, 0.f);
    u_lo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    set_error(err, ERR_BAD_SAMPLE);
    return;
  }
  df32 sb, cb, sl, cl;
  df_sincos_deg(la, sb, cb);
  df_sincos_deg(lo, sl, cl);
  key[i] = (uint32_t)ang2pix_ring_dual(ns, lo, la, sb);
  const df32 x = df_mul(cb, cl), y = df_mul(cb, sl);
  float w = 1.f;
  if (weights) {
    w = weights[i];
    if (!(w >= 0.f) || !isfinite(w)) {
      set_error(err, ERR_BAD_SAMPLE);
      w = 0.f;
    }
  }
  u_hi[i] = make_float4(x.hi, y.hi, sb.hi, w);
  u_lo[i] = make_float4(x.lo, y.lo, sb.lo, 0.f);
}

// Ring number of pixel p (RING scheme); the belt division by 4 ns is a
// shift when nside is a power of two (log2 given, else -1).
__device__ __forceinline__ int64_t ring_of_key(int64_t ns, int lg, int64_t p) {
  const int64_t ncap = 2 * ns * (ns - 1);
  if (p >= ncap && p < 12 * ns * ns - ncap)
    return ns + (lg >= 0 ? ((p - ncap) >> (lg + 2)) : (p - ncap) / (4 * ns));
  return ring_of_pix(ns, p);
}

// Sorted order: gather the unit vectors, and ring_off[i] = first sorted
// position with ring >= i, i = 0 .. 4 ns (thread s writes the entries for
// the rings after its predecessor's ring up to its own).
__global__ void k_sample_gather(int64_t ns, int lg, const uint32_t* __restrict__ skey,
                                const uint32_t* __restrict__ sval,
                                const float4* __restrict__ u_hi,
                                const float4* __restrict__ u_lo, int64_t n,
                                float4* __restrict__ s_hi, float4* __restrict__ s_lo,
                                int32_t* __restrict__ ring_off) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t npix = 12 * ns * ns;
  const int64_t end = 4 * ns;
  int64_t rc = end;
  if (s < n) {
    const uint32_t idx = sval[s];
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

__device__ __forceinline__ int32_t lower_bound_u32(const uint32_t* __restrict__ a, int32_t lo,
                                                   int32_t hi, uint32_t v) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
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

int key_bits_for(int64_t ns) {
  const uint64_t maxkey = (uint64_t)(12 * ns * ns);  // sentinel for invalid samples
  int b = 0;
  while (b < 32 && (maxkey >> b) != 0) ++b;
  return b;
}

}  // namespace

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
  dfree(t.sub64, s);
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
  const int warps = 8;
  k_tile_query<<<ceil_div(nt, warps), 32 * warps, 0, s>>>(t.c64, t.sub64, nt, g->nside, r,
                                                        counts, nullptr, nullptr, 0);
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
  k_tile_query<<<ceil_div(nt, warps), 32 * warps, 0, s>>>(t.c64, t.sub64, nt, g->nside, r,
                                                        nullptr, t.range_off, t.ranges, 1);
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
  dfree(g->u_hi, s);
  dfree(g->u_lo, s);
  g->cap_n = 0;
  cudaError_t e;
  if ((e = dalloc(&g->key, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->val, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->s_hi, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->s_lo, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->u_hi, (size_t)n, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->u_lo, (size_t)n, s)) != cudaSuccess) return e;
  g->cap_n = (size_t)n;
  return cudaSuccess;
}

cudaError_t samples_keys(cg_grid* g, const double* lon, const double* lat, const float* weights,
                         int64_t n) {
  cudaError_t e = ensure_samples(g, n);
  if (e != cudaSuccess) return e;
  k_sample_keys<<<ceil_div(n, 256), 256, 0, g->stream>>>(g->nside, lon, lat, weights, n, g->key,
                                                         g->val, g->u_hi, g->u_lo, g->d_err);
  g->n_launches += 1;
  return cudaGetLastError();
}

cudaError_t samples_sort(cg_grid* g, int64_t n) {
  const int bits = key_bits_for(g->nside);
  g->n_launches += 3 * ((bits + 7) / 8);
  return radix_sort_u32(g->key, g->val, n, bits, g->sw, g->stream, &g->sorted_key,
                        &g->sorted_val);
}

cudaError_t samples_prepare(cg_grid* g, const double* lon, const double* lat,
                            const float* weights, int64_t n, Tiling& t) {
  cudaStream_t s = g->stream;
  const int64_t ns = g->nside;
  int lg = -1;
  if ((ns & (ns - 1)) == 0)
    for (lg = 0; ((int64_t)1 << lg) < ns; ++lg) {
    }
  k_sample_gather<<<ceil_div(n + 1, 256), 256, 0, s>>>(ns, lg, g->sorted_key, g->sorted_val,
                                                       g->u_hi, g->u_lo, n, g->s_hi, g->s_lo,
                                                       g->ring_off);
  g->n_launches += 1;
  if (t.n_tiles > 0) {
    const int warps = 8;
    k_tile_ranges<<<ceil_div(t.n_tiles, warps), 32 * warps, 0, s>>>(
        t.ranges, t.range_off, t.n_tiles, g->ring_off, g->sorted_key, t.range_s, t.range_c,
        t.tile_cand);
    g->n_launches += 1;
  }
  g->last_n = n;
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
