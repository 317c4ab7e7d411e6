// cg_common.cuh -- device helpers shared by the gridding kernels.
//
// Precision plan (GB300 runs FP64 at ~1/70 of FP32, so FP64 is kept off the
// per-pair path):
//   * per sample / per target: unit vectors carried as double-float (hi, lo)
//     pairs of FP32, so differences of nearby vectors keep ~47 bits;
//   * per (target, candidate) pair: FP32 arithmetic on tile-relative vectors;
//   * FP64 only for the HEALPix index (mirroring the reference definition
//     operation by operation) and for the rare pairs whose support cut lies
//     inside a guard band around d = r.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

// Device error word bits.
enum : unsigned {
  ERR_BAD_SAMPLE = 1u,   // non-finite or out-of-range sample coordinate
  ERR_BAD_TARGET = 2u,   // non-finite or out-of-range target coordinate
  ERR_INTERNAL = 4u,     // an internal bound was exceeded
  ERR_TIMEOUT = 8u,      // a bounded wait gave up
};

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg2Rad = (3.14159265358979323846 / 180.0);

__device__ __forceinline__ void set_error(unsigned* err, unsigned bit) {
  if (err) atomicOr(err, bit);
}

// sin(pi x) / (pi x), 1 at x = 0 (the tapered-sinc kernel's sinc factor)
__device__ __forceinline__ float sinc_pi(float x) {
  return (x == 0.f) ? 1.f : sinpif(x) / (3.14159265358979f * x);
}

// ---------------------------------------------------------------------------
// HEALPix RING index in FP64 (Gorski et al. 2005; the paper's Sect. 2.2
// step 3a).  The operation sequence is fixed with explicit round-to-nearest
// intrinsics (no FMA contraction) so that it reproduces the plain FP64
// definition bit for bit except where sin() itself differs in the last ulp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lon_fold_deg(double lon) {
  double p = lon;
  if (!(p >= 0.0 && p < 360.0)) {
    p = __dsub_rn(p, __dmul_rn(360.0, floor(__ddiv_rn(p, 360.0))));
    if (p >= 360.0) p = __dsub_rn(p, 360.0);
    if (p < 0.0) p = 0.0;
  }
  return p;
}

__device__ __forceinline__ int64_t ang2pix_ring_f64(int64_t ns, double lon_deg, double lat_deg) {
  const double z = sin(__dmul_rn(lat_deg, kDeg2Rad));
  const double za = fabs(z);
  const double phi = lon_fold_deg(lon_deg);
  const double tt = __ddiv_rn(phi, 90.0);
  const double dns = (double)ns;
  if (za <= 2.0 / 3.0) {
    // belt: diamonds between ascending and descending edge lines
    const double u = __dmul_rn(dns, __dadd_rn(0.5, tt));
    const double v = __dmul_rn(dns, __dmul_rn(z, 0.75));
    const int64_t asc = (int64_t)__dsub_rn(u, v);
    const int64_t dsc = (int64_t)__dadd_rn(u, v);
    int64_t k = ns + 1 + asc - dsc;
    // a point on the boundary ring |z| = 2/3 at a pixel-corner longitude can
    // round to ring 0 or 2 ns + 2, outside the belt: it belongs to the
    // boundary ring (belt rings are 1 .. 2 ns + 1)
    k = k < 1 ? 1 : (k > 2 * ns + 1 ? 2 * ns + 1 : k);
    const int64_t odd = k & 1;
    int64_t j = (asc + dsc - ns + (1 - odd) + 1) / 2;
    j %= 4 * ns;
    if (j < 0) j += 4 * ns;
    return 2 * ns * (ns - 1) + (k - 1) * 4 * ns + j;
  } else {
    // polar caps: ring counted from the pole = sum of the two edge indices + 1
    const double t = __dsub_rn(tt, floor(tt));
    const double x = __dmul_rn(dns, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
    const int64_t a = (int64_t)__dmul_rn(t, x);
    const int64_t b = (int64_t)__dmul_rn(__dsub_rn(1.0, t), x);
    int64_t k = a + b + 1;
    if (k > ns) k = ns;   // the same boundary: cap rings are 1 .. ns
    int64_t j = (int64_t)__dmul_rn(tt, (double)k);
    j %= 4 * k;
    if (j < 0) j += 4 * k;
    if (z > 0.0) return 2 * k * (k - 1) + j;
    return 12 * ns * ns - 2 * k * (k + 1) + j;
  }
}

// Ring number (1 .. 4ns-1) of RING pixel p; integer arithmetic with an
// FP32 square-root estimate corrected exactly.
__device__ __forceinline__ int ring_of_pix(int64_t ns, int64_t p) {
  const int64_t npix = 12 * ns * ns;
  const int64_t ncap = 2 * ns * (ns - 1);
  if (p < ncap) {
    int64_t k = (int64_t)(0.5f * (1.0f + sqrtf(1.0f + 2.0f * (float)p)));
    while (k > 1 && 2 * k * (k - 1) > p) --k;
    while (2 * (k + 1) * k <= p) ++k;
    return (int)k;
  }
  if (p < npix - ncap) return (int)(ns + (p - ncap) / (4 * ns));
  const int64_t q = npix - 1 - p;
  int64_t k = (int64_t)(0.5f * (1.0f + sqrtf(1.0f + 2.0f * (float)q)));
  while (k > 1 && 2 * k * (k - 1) > q) --k;
  while (2 * (k + 1) * k <= q) ++k;
  return (int)(4 * ns - k);
}

// ---------------------------------------------------------------------------
// double-float helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// Difference of two double-float values as one float: (ah + al) - (bh + bl).
// For nearby values ah - bh is exact (Sterbenz) or tiny, so the result keeps
// full FP32 relative precision of the difference itself.
__device__ __forceinline__ float df_diff(float ah, float al, float bh, float bl) {
  return (ah - bh) + (al - bl);
}

}  // namespace cg
