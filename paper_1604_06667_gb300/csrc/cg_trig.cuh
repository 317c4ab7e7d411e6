// cg_trig.cuh -- sine and cosine of an FP64 angle in degrees as double-float
// (hi, lo) FP32 pairs, on the FP32 pipes.
//
// GB300 runs FP64 at ~1/70 of the FP32 rate, and a sample needs four
// trigonometric values for its unit vector (cos b cos l, cos b sin l, sin b)
// and its HEALPix index (z = sin b).  Method: table-driven argument reduction
// with the angle-addition formula (Tang's table method):
//   a = r + 90 n                  (exact in FP64, |r| <= 45 deg)
//   x = r pi / 180 = j / 64 + t   (double-float, |t| <= 1/128)
//   sin x = S_j cos t + C_j sin t,  cos x = C_j cos t - S_j sin t
// with S_j = sin(j/64), C_j = cos(j/64) tabulated as double-float and
// cos t = 1 - (t^2/2 - t^4/24), sin t = t - t (t^2/6 - t^4/120) (Taylor; the
// next terms are below 4e-16).  Absolute error ~1e-14, far below what the
// tile-relative FP32 vectors built from these values can resolve (~5e-10).
// The table is computed at compile time from the Taylor series in FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df32{s, e};
}
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return df32{s, b - (s - a)};
}
__device__ __forceinline__ df32 df_two_prod(float a, float b) {
  const float p = a * b;
  return df32{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  const df32 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const df32 p = df_two_prod(a.hi, b.hi);
  return df_fast_two_sum(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}
__device__ __forceinline__ df32 df_neg(df32 a) { return df32{-a.hi, -a.lo}; }

// ---- table S_j, C_j, j = 0 .. kTrigTab - 1, at j / 64 rad -------------------
constexpr int kTrigTab = 53;   // covers |x| <= pi/4 + margin (52 / 64 = 0.8125)

constexpr double trig_taylor(double x, bool sine) {
  // alternating series; 24 terms are exact to FP64 rounding for |x| < 1
  double term = sine ? x : 1.0;
  double sum = term;
  int k = sine ? 1 : 0;
  for (int i = 0; i < 24; ++i) {
    term = -term * x * x / (double)((k + 1) * (k + 2));
    k += 2;
    sum += term;
  }
  return sum;
}

struct alignas(16) TrigTable {
  float v[kTrigTab * 4];   // S_hi, S_lo, C_hi, C_lo
  constexpr TrigTable() : v() {
    for (int j = 0; j < kTrigTab; ++j) {
      const double x = (double)j / 64.0;
      const double s = trig_taylor(x, true), c = trig_taylor(x, false);
      const float sh = (float)s, ch = (float)c;
      v[4 * j + 0] = sh;
      v[4 * j + 1] = (float)(s - (double)sh);
      v[4 * j + 2] = ch;
      v[4 * j + 3] = (float)(c - (double)ch);
    }
  }
};

__device__ constexpr TrigTable kTrigTable{};

// pi / 180 as double-float
constexpr double kD2R = 3.14159265358979323846 / 180.0;
constexpr float kD2R_hi = (float)kD2R;
constexpr float kD2R_lo = (float)(kD2R - (double)kD2R_hi);

// sin and cos of a (degrees, finite, |a| < 2^40).
__device__ __forceinline__ void df_sincos_deg(double a, df32& s, df32& c) {
  const double qd = rint(a * (1.0 / 90.0));
  const double r = fma(-90.0, qd, a);      // exact: 90 qd and a share the grid of a
  const int n = (int)((int64_t)qd & 3);
  const float rh = __double2float_rn(r);
  const float rl = __double2float_rn(r - (double)rh);
  const df32 x = df_mul(df32{rh, rl}, df32{kD2R_hi, kD2R_lo});
  const int j = __float2int_rn(x.hi * 64.f);
  const int ja = j < 0 ? -j : j;
  const float4 tab = *reinterpret_cast<const float4*>(&kTrigTable.v[4 * ja]);
  const df32 S = (j < 0) ? df32{-tab.x, -tab.y} : df32{tab.x, tab.y};
  const df32 C = df32{tab.z, tab.w};
  const df32 t = df_two_sum(x.hi - (float)j * (1.f / 64.f), x.lo);   // first term exact
  // t^2 as double-float, u = t^2/2 - t^4/24 = 1 - cos t
  const df32 t2 = df_two_prod(t.hi, t.hi);
  const float t2lo = fmaf(2.f * t.hi, t.lo, t2.lo);
  const df32 u = df_fast_two_sum(0.5f * t2.hi, fmaf(-t2.hi * (1.f / 24.f), t2.hi, 0.5f * t2lo));
  // sin t = t - t v, v = t^2/6 - t^4/120
  const float v = t2.hi * fmaf(-t2.hi, 1.f / 120.f, 1.f / 6.f);
  const df32 st = df_add(t, df32{-t.hi * v, -t.lo * v});
  // sin x = S - S u + C sin t ;  cos x = C - C u - S sin t
  const df32 sx = df_add(df_add(S, df_neg(df_mul(S, u))), df_mul(C, st));
  const df32 cx = df_add(df_add(C, df_neg(df_mul(C, u))), df_neg(df_mul(S, st)));
  // rotate by the quadrant n: a = r + 90 n
  switch (n) {
    case 0: s = sx; c = cx; break;
    case 1: s = cx; c = df_neg(sx); break;
    case 2: s = df_neg(sx); c = df_neg(cx); break;
    default: s = df_neg(cx); c = sx; break;
  }
}

// ---- the same without FP64 arithmetic -------------------------------------
// GB300 executes FP64 (and FP64 <-> FP32 conversions) at a few operations per
// SM and clock, so the per-sample path splits its FP64 inputs with integer
// operations and reduces the argument in double-float.

// a as hi + lo: hi = a truncated to 24 significant bits, lo = the remainder
// rounded to FP32 (|error| <= 2^-48 |a|).  Valid for 2^-100 <= |a| < 2^100 or
// a = 0 (df_split_ok tells).
__device__ __forceinline__ bool df_split_ok(double a) {
  const int e = (int)((__double_as_longlong(a) >> 52) & 0x7ff);
  return e == 0 ? a == 0.0 : (e >= 1023 - 100 && e < 1023 + 100);
}
__device__ __forceinline__ df32 df_split(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return df32{0.f, 0.f};
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  // remainder: the low 29 mantissa bits, worth 2^(e - 1075) each
  const float r = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull));
  const float scale = __uint_as_float((unsigned)(e - 1023 - 23 + 127) << 23);   // 2^(e-1046)
  const float lo = r * 1.86264514923095703125e-9f * scale;                       // r 2^-29 2^(e-1046)
  return df32{hi, sign ? -lo : lo};
}

// sin and cos of a (degrees, double-float, |a| < 2^17): as df_sincos_deg with
// the reduction a = r + 90 n done in double-float (90 n is exact in FP32).
__device__ __forceinline__ void df_sincos_deg_df(df32 a, df32& s, df32& c) {
  const float qd = rintf(a.hi * (1.f / 90.f));
  const df32 r = df_add(a, df32{-90.f * qd, 0.f});    // |r| <= 45 deg (+ rounding)
  const int n = (int)qd & 3;
  const df32 x = df_mul(r, df32{kD2R_hi, kD2R_lo});
  const int j = __float2int_rn(x.hi * 64.f);
  const int ja = j < 0 ? -j : j;
  const float4 tab = *reinterpret_cast<const float4*>(&kTrigTable.v[4 * ja]);
  const df32 S = (j < 0) ? df32{-tab.x, -tab.y} : df32{tab.x, tab.y};
  const df32 C = df32{tab.z, tab.w};
  const df32 t = df_two_sum(x.hi - (float)j * (1.f / 64.f), x.lo);
  const df32 t2 = df_two_prod(t.hi, t.hi);
  const float t2lo = fmaf(2.f * t.hi, t.lo, t2.lo);
  const df32 u = df_fast_two_sum(0.5f * t2.hi, fmaf(-t2.hi * (1.f / 24.f), t2.hi, 0.5f * t2lo));
  const float v = t2.hi * fmaf(-t2.hi, 1.f / 120.f, 1.f / 6.f);
  const df32 st = df_add(t, df32{-t.hi * v, -t.lo * v});
  const df32 sx = df_add(df_add(S, df_neg(df_mul(S, u))), df_mul(C, st));
  const df32 cx = df_add(df_add(C, df_neg(df_mul(C, u))), df_neg(df_mul(S, st)));
  switch (n) {
    case 0: s = sx; c = cx; break;
    case 1: s = cx; c = df_neg(sx); break;
    case 2: s = df_neg(sx); c = df_neg(cx); break;
    default: s = df_neg(cx); c = sx; break;
  }
}

}  // namespace cg
