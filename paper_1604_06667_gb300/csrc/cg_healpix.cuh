// cg_healpix.cuh -- device-side HEALPix RING geometry shared by the sample
// index (k_healpix.cu) and the degridder's target index (k_degrid.cu):
// ring geometry, the closed-form pixel intervals of a disc on a ring (the
// per-ring treatment of the paper's Sect. 3.3), the RING index of a sample
// from its double-float sine with exact FP64 fallback, and binary search.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

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
    if (discs[q].R < 0.0) continue;   // empty group
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
    // near a pole sqrt(1 - za) magnifies the error of z (<= 1e-13): with
    // 1 - za > 1e-5 the error of x stays below 0.5e-13 nside sqrt(3) /
    // sqrt(1e-5) < 5e-7 for nside <= 16384, inside the margin; nearer the
    // pole FP64 decides
    good = good && ft > 1e-12 && ft < 1.0 - 1e-12 && 1.0 - za > 1e-5;
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

// floor of a double-float and its fractional part (as FP32).
__device__ __forceinline__ float df_floor(df32 a, float& frac) {
  float f = floorf(a.hi);
  if (f == a.hi && a.lo < 0.f) f -= 1.f;   // a sits just below the integer a.hi
  frac = (a.hi - f) + a.lo;                 // a.hi - f is exact
  return f;
}

// ang2pix_ring_fast in double-float arithmetic (no FP64 operations):
// longitude lon (degrees, double-float, folded here), z = sin lat as a
// double-float (|error| ~1e-14).  *ok = false near the cap/belt boundary
// (| |z| - 2/3 | <= 1e-6), within 1e-5 of a pole's z, at a quadrant boundary
// of the caps, or when a truncated quantity lies within the 1e-6 margin of an
// integer: df32 evaluates the truncated quantities (at most 4 nside = 65536)
// to ~1e-8 absolute, so the decisions outside the margin are those of the
// FP64 definition.
__device__ __forceinline__ int64_t ang2pix_ring_df(int64_t ns, df32 lon, df32 z, bool* ok) {
  constexpr float M = 1e-6f;
  constexpr float kZb = (float)(2.0 / 3.0);
  const float za = fabsf(z.hi);
  const bool belt = za < kZb - 1e-6f;
  if (!(belt || (za > kZb + 1e-6f && za < 1.f - 1e-5f)) || ns > 16384) {
    *ok = false;
    return 0;
  }
  // phi in [0, 360): fold by whole turns (exact in FP32 for |lon| < 2^24)
  if (lon.hi < 0.f || lon.hi >= 360.f) {
    const float k = floorf(lon.hi * (1.f / 360.f));
    lon = df_add(lon, df32{-360.f * k, 0.f});
    if (lon.hi < 0.f) lon = df_add(lon, df32{360.f, 0.f});
    if (lon.hi >= 360.f) lon = df_add(lon, df32{-360.f, 0.f});
  }
  constexpr double kInv90 = 1.0 / 90.0;
  const df32 tt = df_mul(lon, df32{(float)kInv90, (float)(kInv90 - (double)(float)kInv90)});
  const float dns = (float)ns;                           // exact: ns <= 16384
  if (belt) {
    // diamonds between ascending and descending edge lines
    const df32 u = df_mul(df_add(tt, df32{0.5f, 0.f}), df32{dns, 0.f});
    const df32 v = df_mul(z, df32{0.75f * dns, 0.f});
    const df32 A = df_add(u, df_neg(v)), B = df_add(u, v);
    float fa, fb;
    const float Af = df_floor(A, fa), Bf = df_floor(B, fb);
    *ok = fa > M && fa < 1.f - M && fb > M && fb < 1.f - M;
    const int64_t asc = (int64_t)Af;
    const int64_t dsc = (int64_t)Bf;
    int64_t k = ns + 1 + asc - dsc;
    k = k < 1 ? 1 : (k > 2 * ns + 1 ? 2 * ns + 1 : k);
    const int64_t odd = k & 1;
    int64_t j = (asc + dsc - ns + (1 - odd) + 1) / 2;
    j %= 4 * ns;
    if (j < 0) j += 4 * ns;
    return 2 * ns * (ns - 1) + (k - 1) * 4 * ns + j;
  }
  // polar caps: ring counted from the pole = sum of the two edge indices + 1,
  // the edge indices from the fraction ft of the quadrant and
  // x = nside sqrt(3 (1 - |z|))
  float ftf;
  const float tf = df_floor(tt, ftf);
  const df32 ft = df_add(tt, df32{-tf, 0.f});             // tt - floor(tt), as a double-float
  const df32 omft = df_add(df32{1.f, 0.f}, df_neg(ft));
  const df32 zabs = z.hi < 0.f ? df_neg(z) : z;
  const df32 w = df_mul(df32{3.f, 0.f}, df_add(df32{1.f, 0.f}, df_neg(zabs)));
  // square root: FP32 estimate and one Newton step on the double-float residual
  const float s0 = sqrtf(w.hi);
  const df32 res = df_add(w, df_neg(df_two_prod(s0, s0)));
  const df32 sq = df_fast_two_sum(s0, res.hi * (0.5f / s0));
  const df32 x = df_mul(sq, df32{dns, 0.f});
  const df32 P = df_mul(ft, x), Q = df_mul(omft, x);
  float fp, fq;
  const float Pf = df_floor(P, fp), Qf = df_floor(Q, fq);
  bool good = ft.hi > 1e-12f && omft.hi > 1e-12f;
  good = good && fp > M && fp < 1.f - M && fq > M && fq < 1.f - M;
  const int64_t k = (int64_t)Pf + (int64_t)Qf + 1;
  const df32 J = df_mul(tt, df32{(float)k, 0.f});           // k <= nside: exact in FP32
  float fj;
  const float Jf = df_floor(J, fj);
  *ok = good && fj > M && fj < 1.f - M;
  int64_t j = (int64_t)Jf;
  j %= 4 * k;
  if (j < 0) j += 4 * k;
  return (z.hi > 0.f) ? 2 * k * (k - 1) + j : 12 * ns * ns - 2 * k * (k + 1) + j;
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

// Ring number of pixel p (RING scheme); the belt division by 4 ns is a
// shift when nside is a power of two (log2 given, else -1).
__device__ __forceinline__ int64_t ring_of_key(int64_t ns, int lg, int64_t p) {
  const int64_t ncap = 2 * ns * (ns - 1);
  if (p >= ncap && p < 12 * ns * ns - ncap)
    return ns + (lg >= 0 ? ((p - ncap) >> (lg + 2)) : (p - ncap) / (4 * ns));
  return ring_of_pix(ns, p);
}

__device__ __forceinline__ int32_t lower_bound_u32(const uint32_t* __restrict__ a, int32_t lo,
                                                   int32_t hi, uint32_t v) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace
}  // namespace cg
