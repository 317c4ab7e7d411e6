// cg_cut.cuh -- the support cut d <= r (paper Eq. 3: the kernel is truncated
// at the support radius) for the rare pairs whose FP32 chord fell inside the
// guard band around r.
//
// The FP32 per-pair chord decides every pair outside a band of +-1e-5
// (relative, on chord^2) around the support chord.  Inside it the decision is
// taken again, in two steps: the squared chord of the two double-float unit
// vectors (each component within ~2e-14 of its exact value, so the squared
// chord within ~1.4e-13 x chord) against the FP64 squared chord of r, and,
// only where that difference is within its tolerance (1e-9 relative plus
// 1e-12 x chord), the FP64 haversine distance against r itself.  The first
// step runs on the FP32 pipes (~150 instructions); the second costs thousands
// of cycles of FP64 transcendental work and is reached about once per 10^4
// band pairs.
#pragma once
#include "cg_common.cuh"
#include "cg_trig.cuh"

namespace cg {
namespace {

// Great-circle distance by the haversine formula, FP64.
__device__ __noinline__ double cut_haversine_f64(double l1, double b1, double l2, double b2) {
  const double p1 = b1 * kDeg2Rad, p2 = b2 * kDeg2Rad;
  const double dl = (l2 - l1) * kDeg2Rad;
  const double sdp = sin(0.5 * (p2 - p1));
  const double sdl = sin(0.5 * dl);
  double h = sdp * sdp + cos(p1) * cos(p2) * sdl * sdl;
  h = fmin(h, 1.0);
  return 2.0 * asin(sqrt(h));
}

// Unit vector (cos b cos l, cos b sin l, sin b) of (l, b) in degrees, as
// double-float pairs.
__device__ __forceinline__ void df_unit_vector(double lon, double lat, df32& x, df32& y, df32& z) {
  df32 sb, cb, sl, cl;
  df_sincos_deg(lat, sb, cb);
  df_sincos_deg(lon, sl, cl);
  x = df_mul(cb, cl);
  y = df_mul(cb, sl);
  z = sb;
}

// Is the pair (target (lon, lat) tl, sample sl, degrees) within the support?
// c2r_hi + c2r_lo: FP64 squared chord of r as a double-float; c2r_tol: the
// tolerance of the double-float squared chord (see above); r_rad: r.
__device__ __forceinline__ bool pair_inside_inl(double2 tl, double2 sl, float c2r_hi,
                                                float c2r_lo, float c2r_tol, double r_rad) {
  df32 tx, ty, tz, sx, sy, sz;
  df_unit_vector(tl.x, tl.y, tx, ty, tz);
  df_unit_vector(sl.x, sl.y, sx, sy, sz);
  const df32 dx = df_add(tx, df_neg(sx));
  const df32 dy = df_add(ty, df_neg(sy));
  const df32 dz = df_add(tz, df_neg(sz));
  const df32 c2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
  const df32 diff = df_add(c2, df32{-c2r_hi, -c2r_lo});
  if (diff.hi > c2r_tol) return false;
  if (diff.hi < -c2r_tol) return true;
  return cut_haversine_f64(tl.x, tl.y, sl.x, sl.y) <= r_rad;
}

// The same decision out of line (for call sites inside loops whose
// registers it should not inflate).
__device__ __noinline__ bool pair_inside(double2 tl, double2 sl, float c2r_hi, float c2r_lo,
                                         float c2r_tol, double r_rad) {
  return pair_inside_inl(tl, sl, c2r_hi, c2r_lo, c2r_tol, r_rad);
}

}  // namespace
}  // namespace cg
