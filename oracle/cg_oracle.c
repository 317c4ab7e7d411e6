/*
 * cg_oracle.c -- plain FP64 CPU oracle for convolution-based gridding.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * Every routine is written for obviousness, not speed:
 *   - all arithmetic in IEEE binary64, compiled without FMA contraction;
 *   - sums that feed a comparison use Neumaier-compensated accumulation;
 *   - no blocking, fusion or reordering beyond what the definition states.
 *
 * Paper: Winkel, Lenz & Floeer, "Cygrid: A fast Cython-powered
 * convolution-based gridding module for Python" (A&A 2016, arXiv 1604.06667).
 *   Eq. 1  unnormalised kernel sum          -> grid_* numerator
 *   Eq. 2  weight map                        -> grid_* weight sum
 *   Eq. 3  normalised map                    -> grid_* output
 *   Sect. 2.1 enumerate (zero, accumulate, divide) -> brute-force gridder
 *   Sect. 2.2 steps 1-3c (HEALPix lookup)    -> lookup gridder
 *   Sect. 3.3 query-disk (Eq. 4-5)           -> query_disc / ring shift
 *   Sect. 3.5 kernel, support radius, hpx-max-resolution -> kernel + nside rule
 * HEALPix geometry follows Gorski et al. (2005, ApJ 622, 759), which the
 * paper cites for the tessellation (Sect. 2.2, 3.2).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - gauss1d: w(d) = exp(-d^2 / (2 sigma^2)), unnormalised (Eq. 3 makes the
 *     normalisation irrelevant).
 *   - elliptical Gaussian: bearing beta of the sample seen from the target,
 *     measured from north through east; a = d cos(beta-PA), b = d sin(beta-PA),
 *     w = exp(-a^2/(2 smaj^2) - b^2/(2 smin^2)).
 *   - support: closed cut d <= r.
 *   - per-sample weight omega_n multiplies both the numerator and W.
 *   - W == 0 -> output NaN.
 *   - longitude normalisation phi = lon mod 360 in [0,360); theta = 90 - lat.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_DEG2RAD (OR_PI / 180.0)

/* ------------------------------------------------------------------------ */
/* Neumaier compensated accumulator                                          */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } or_acc;

static void acc_add(or_acc* a, double x) {
  double t = a->s + x;
  /* the correction term is defined for finite sums only; once a term is
   * infinite or NaN the sum is that of plain IEEE summation (Eq. 1 with such a
   * value: +-Inf, or NaN for Inf - Inf or a NaN term) */
  if (isfinite(t)) {
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
  }
  a->s = t;
}
static double acc_get(const or_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Input angle conventions                                                   */
/* ------------------------------------------------------------------------ */

/* Longitude in degrees folded into [0, 360). */
double or_lon_fold_deg(double lon) {
  double p = lon;
  if (!(p >= 0.0 && p < 360.0)) {
    p = p - 360.0 * floor(p / 360.0);
    if (p >= 360.0) p = p - 360.0;
    if (p < 0.0) p = 0.0;
  }
  return p;
}

/* ------------------------------------------------------------------------ */
/* HEALPix RING scheme (Gorski et al. 2005; paper Sect. 2.2, 3.2, 3.3)       */
/*                                                                           */
/* Rings are numbered i = 1 .. 4*nside-1 from the north pole.  Rings 1..ns-1 */
/* form the north polar cap (ring i holds 4i pixels at z = 1 - i^2/(3ns^2)), */
/* rings ns..3ns the equatorial belt (4ns pixels each, z = 4/3 - 2i/(3ns)),  */
/* and the rest mirror the north cap.  Pixel indices run ring by ring from   */
/* the north pole, eastwards from phi = 0 within a ring.                     */
/* ------------------------------------------------------------------------ */

/* Pixel index of direction (lon, lat) in degrees.  Belt: the pixel is the
 * diamond cut out by two families of straight lines in (phi, z), the
 * "ascending" lines u - v = const and the "descending" lines u + v = const
 * with u = ns*(1/2 + phi/(pi/2)) and v = (3/4)*ns*z; their integer parts
 * name the diamond.  Caps: with x = ns*sqrt(3(1-|z|)) and the fractional
 * quadrant position t, the lines t*x = const and (1-t)*x = const play the
 * same role, and the ring counted from the pole is their sum plus one. */
int64_t or_ang2pix_ring(int64_t ns, double lon_deg, double lat_deg) {
  const double z = sin(lat_deg * OR_DEG2RAD);
  const double za = fabs(z);
  const double phi = or_lon_fold_deg(lon_deg);
  const double tt = phi / 90.0;                 /* quadrant coordinate [0,4) */
  const double dns = (double)ns;
  if (za <= 2.0 / 3.0) {
    const double u = dns * (0.5 + tt);
    const double v = dns * (z * 0.75);
    const int64_t asc = (int64_t)(u - v);       /* ascending line index  */
    const int64_t dsc = (int64_t)(u + v);       /* descending line index */
    int64_t k = ns + 1 + asc - dsc;             /* belt ring from z=2/3, 1..2ns+1 */
    /* a point on the boundary ring |z| = 2/3 whose longitude is a pixel
     * corner can round to ring 0 or 2ns+2, outside the belt: it belongs to
     * the boundary ring (Gorski et al. 2005: belt rings are 1 .. 2ns+1) */
    if (k < 1) k = 1;
    if (k > 2 * ns + 1) k = 2 * ns + 1;
    const int64_t odd = k & 1;
    int64_t j = (asc + dsc - ns + (1 - odd) + 1) / 2;
    j = j % (4 * ns);
    if (j < 0) j += 4 * ns;
    return 2 * ns * (ns - 1) + (k - 1) * 4 * ns + j;
  } else {
    const double t = tt - floor(tt);            /* position inside quadrant */
    const double x = dns * sqrt(3.0 * (1.0 - za));
    const int64_t a = (int64_t)(t * x);
    const int64_t b = (int64_t)((1.0 - t) * x);
    int64_t k = a + b + 1;                      /* ring counted from the pole */
    if (k > ns) k = ns;                         /* the same boundary: cap rings 1 .. ns */
    int64_t j = (int64_t)(tt * (double)k);
    j = j % (4 * k);
    if (j < 0) j += 4 * k;
    if (z > 0.0) return 2 * k * (k - 1) + j;
    return 12 * ns * ns - 2 * k * (k + 1) + j;
  }
}

void or_ang2pix_ring_many(int64_t ns, int64_t n, const double* lon, const double* lat,
                          int64_t* pix) {
  for (int64_t i = 0; i < n; ++i) pix[i] = or_ang2pix_ring(ns, lon[i], lat[i]);
}

/* Smallest distance, in the units of the floored quantities, between any
 * quantity that ang2pix truncates and the nearest integer; also covers the
 * cap/belt switch |z| = 2/3.  A sample with a tiny margin sits on a pixel
 * boundary, where FP64 rounding differences between two correct
 * implementations may pick either neighbour. */
double or_ang2pix_margin(int64_t ns, double lon_deg, double lat_deg) {
  const double z = sin(lat_deg * OR_DEG2RAD);
  const double za = fabs(z);
  const double phi = or_lon_fold_deg(lon_deg);
  const double tt = phi / 90.0;
  const double dns = (double)ns;
  double m = fabs(za - 2.0 / 3.0) * dns;
  double q[3];
  int nq = 0;
  if (za <= 2.0 / 3.0) {
    const double u = dns * (0.5 + tt);
    const double v = dns * (z * 0.75);
    q[nq++] = u - v;
    q[nq++] = u + v;
  } else {
    const double t = tt - floor(tt);
    const double x = dns * sqrt(3.0 * (1.0 - za));
    q[nq++] = t * x;
    q[nq++] = (1.0 - t) * x;
    const int64_t k = (int64_t)(t * x) + (int64_t)((1.0 - t) * x) + 1;
    q[nq++] = tt * (double)k;
    /* quadrant boundary (t wraps) */
    double e = fabs(tt - floor(tt + 0.5)) * dns;
    if (e < m) m = e;
  }
  for (int i = 0; i < nq; ++i) {
    double e = fabs(q[i] - floor(q[i] + 0.5));
    if (e < m) m = e;
  }
  return m;
}

/* Ring geometry: for ring i (1..4ns-1) the pixel count, first pixel index,
 * centre z, and the phase of the first pixel centre in units of the pixel
 * spacing (phi_j = (j + phase) * 2 pi / count). */
void or_ring_info(int64_t ns, int64_t i, int64_t* count, int64_t* first, double* z,
                  double* phase) {
  const int64_t npix = 12 * ns * ns;
  const double dns = (double)ns;
  if (i < ns) {
    *count = 4 * i;
    *first = 2 * i * (i - 1);
    *z = 1.0 - (double)(i * i) / (3.0 * dns * dns);
    *phase = 0.5;
  } else if (i <= 3 * ns) {
    *count = 4 * ns;
    *first = 2 * ns * (ns - 1) + (i - ns) * 4 * ns;
    *z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * dns);
    /* rings with (i - ns) even carry a half-pixel phase */
    *phase = ((i - ns) % 2 == 0) ? 0.5 : 0.0;
  } else {
    const int64_t k = 4 * ns - i;
    *count = 4 * k;
    *first = npix - 2 * k * (k + 1);
    *z = -(1.0 - (double)(k * k) / (3.0 * dns * dns));
    *phase = 0.5;
  }
}

/* Ring number (1..4ns-1) holding pixel p. */
int64_t or_pix2ring(int64_t ns, int64_t p) {
  const int64_t npix = 12 * ns * ns;
  const int64_t ncap = 2 * ns * (ns - 1);
  if (p < ncap) {
    /* ring k holds [2k(k-1), 2k(k+1)) */
    int64_t k = (int64_t)floor(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)p)));
    while (k > 1 && 2 * k * (k - 1) > p) --k;
    while (2 * (k + 1) * k <= p) ++k;
    return k;
  }
  if (p < npix - ncap) return ns + (p - ncap) / (4 * ns);
  {
    const int64_t q = npix - 1 - p;
    int64_t k = (int64_t)floor(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)q)));
    while (k > 1 && 2 * k * (k - 1) > q) --k;
    while (2 * (k + 1) * k <= q) ++k;
    return 4 * ns - k;
  }
}

/* Centre of pixel p: z = cos(theta) and phi in radians [0, 2 pi). */
void or_pix2ang_ring(int64_t ns, int64_t p, double* z, double* phi) {
  int64_t count, first;
  double phase;
  const int64_t i = or_pix2ring(ns, p);
  or_ring_info(ns, i, &count, &first, z, &phase);
  *phi = ((double)(p - first) + phase) * (2.0 * OR_PI / (double)count);
}

/* Colatitude (radians) of the centre of ring i, with the poles as rings 0
 * and 4ns. */
static double ring_theta(int64_t ns, int64_t i) {
  int64_t count, first;
  double z, phase;
  if (i <= 0) return 0.0;
  if (i >= 4 * ns) return OR_PI;
  or_ring_info(ns, i, &count, &first, &z, &phase);
  return acos(z);
}

/* ------------------------------------------------------------------------ */
/* Distances and kernels (Eq. 1, Sect. 2.1)                                 */
/* ------------------------------------------------------------------------ */

/* Great-circle distance in radians by the Haversine formula (Sect. 2.1). */
double or_haversine(double lon1_deg, double lat1_deg, double lon2_deg, double lat2_deg) {
  const double p1 = lat1_deg * OR_DEG2RAD, p2 = lat2_deg * OR_DEG2RAD;
  const double dl = (lon2_deg - lon1_deg) * OR_DEG2RAD;
  const double sdp = sin(0.5 * (p2 - p1));
  const double sdl = sin(0.5 * dl);
  double h = sdp * sdp + cos(p1) * cos(p2) * sdl * sdl;
  if (h > 1.0) h = 1.0;
  return 2.0 * asin(sqrt(h));
}

/* Bearing (radians, from north through east) of point 2 seen from point 1. */
double or_bearing(double lon1_deg, double lat1_deg, double lon2_deg, double lat2_deg) {
  const double p1 = lat1_deg * OR_DEG2RAD, p2 = lat2_deg * OR_DEG2RAD;
  const double dl = (lon2_deg - lon1_deg) * OR_DEG2RAD;
  const double y = sin(dl) * cos(p2);
  const double x = cos(p1) * sin(p2) - sin(p1) * cos(p2) * cos(dl);
  return atan2(y, x);
}

typedef struct {
  int32_t type;         /* 0 = gauss1d, 1 = elliptical gauss2d, 2 = tapered sinc */
  double sigma_deg;     /* gauss1d; tapered sinc: taper width b */
  double smaj_deg;      /* gauss2d major-axis sigma; tapered sinc: first zero a */
  double smin_deg;      /* gauss2d minor-axis sigma */
  double pa_deg;        /* gauss2d position angle of the major axis, N through E */
  double support_deg;   /* support radius r */
} or_kernel;

/* Kernel value for target (lt, bt) and sample (ls, bs); returns 0 and sets
 * *inside = 0 when d > r.  Also returns d in radians. */
static double kernel_eval(const or_kernel* k, double lt, double bt, double ls, double bs,
                          int* inside, double* d_out) {
  const double d = or_haversine(lt, bt, ls, bs);
  const double r = k->support_deg * OR_DEG2RAD;
  *d_out = d;
  if (!(d <= r)) { *inside = 0; return 0.0; }
  *inside = 1;
  if (k->type == 0) {
    const double s = k->sigma_deg * OR_DEG2RAD;
    return exp(-(d * d) / (2.0 * s * s));
  } else if (k->type == 2) {
    /* the sin(x)/x kernel of App. A.1, x = pi d / a, tapered by
     * exp(-d^2 / b^2) so that a finite support suffices */
    const double a = k->smaj_deg * OR_DEG2RAD, b = k->sigma_deg * OR_DEG2RAD;
    const double x = OR_PI * d / a;
    const double sinc = (x == 0.0) ? 1.0 : sin(x) / x;
    return sinc * exp(-(d * d) / (b * b));
  } else {
    const double beta = or_bearing(lt, bt, ls, bs);
    const double pa = k->pa_deg * OR_DEG2RAD;
    const double a = d * cos(beta - pa);
    const double b = d * sin(beta - pa);
    const double s1 = k->smaj_deg * OR_DEG2RAD, s2 = k->smin_deg * OR_DEG2RAD;
    return exp(-(a * a) / (2.0 * s1 * s1) - (b * b) / (2.0 * s2 * s2));
  }
}

double or_kernel_value(const or_kernel* k, double lt, double bt, double ls, double bs) {
  int inside;
  double d;
  return kernel_eval(k, lt, bt, ls, bs, &inside, &d);
}

/* ------------------------------------------------------------------------ */
/* Outputs of a gridding run                                                 */
/* ------------------------------------------------------------------------ */
/* num[P][C]   Eq. 1 numerator  sum_n omega_n w_pn D_nc
 * wsum[P]     Eq. 2 weight map sum_n omega_n w_pn
 * out[P][C]   Eq. 3 map num / wsum, NaN where wsum == 0
 * sabs[P][C]  sum_n omega_n w_pn |D_nc| / wsum (scale for error metrics; may be NULL)
 * npairs      number of (target, sample) pairs with d <= r                  */

static void finish_maps(int64_t P, int32_t C, or_acc* anum, or_acc* aw, or_acc* aabs,
                        double* num, double* wsum, double* out, double* sabs) {
  for (int64_t p = 0; p < P; ++p) {
    const double W = acc_get(&aw[p]);
    if (wsum) wsum[p] = W;
    for (int32_t c = 0; c < C; ++c) {
      const double nv = acc_get(&anum[p * C + c]);
      if (num) num[p * C + c] = nv;
      if (out) out[p * C + c] = (W > 0.0) ? nv / W : NAN;
      if (sabs) sabs[p * C + c] = (W > 0.0) ? acc_get(&aabs[p * C + c]) / W : NAN;
    }
  }
}

/* Brute force: Eq. 1-3 written out, every sample against every target. */
int or_grid_bruteforce(int64_t P, const double* lon_t, const double* lat_t, int64_t N,
                       const double* lon_s, const double* lat_s, int32_t C,
                       const double* data, const double* omega, const or_kernel* k,
                       double* num, double* wsum, double* out, double* sabs,
                       int64_t* npairs) {
  or_acc* anum = (or_acc*)calloc((size_t)(P * C), sizeof(or_acc));
  or_acc* aabs = (or_acc*)calloc((size_t)(P * C), sizeof(or_acc));
  or_acc* aw = (or_acc*)calloc((size_t)P, sizeof(or_acc));
  if (!anum || !aabs || !aw) { free(anum); free(aabs); free(aw); return 1; }
  int64_t pairs = 0;
  for (int64_t p = 0; p < P; ++p) {
    for (int64_t n = 0; n < N; ++n) {
      int inside;
      double d;
      const double w = kernel_eval(k, lon_t[p], lat_t[p], lon_s[n], lat_s[n], &inside, &d);
      if (!inside) continue;
      ++pairs;
      const double ww = w * (omega ? omega[n] : 1.0);
      acc_add(&aw[p], ww);
      for (int32_t c = 0; c < C; ++c) {
        acc_add(&anum[p * C + c], ww * data[n * C + c]);
        acc_add(&aabs[p * C + c], fabs(ww * data[n * C + c]));
      }
    }
  }
  finish_maps(P, C, anum, aw, aabs, num, wsum, out, sabs);
  if (npairs) *npairs = pairs;
  free(anum); free(aabs); free(aw);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* query-disc (Sect. 2.2 step 3b, Sect. 3.3)                                 */
/* ------------------------------------------------------------------------ */
/* Every point of pixel j of ring i lies between the centres of rings i-1 and
 * i+1 in z and within half a pixel spacing (pi / count) of the pixel centre
 * in phi.  The disc query returns every pixel whose such box meets the disc
 * of radius R around (lon, lat): a superset of the pixels that hold a point
 * within R, so an exact distance cut afterwards loses nothing. */

/* Largest phi half-width of the disc over colatitudes [ta, tb]; returns -1
 * if the disc misses the band and a value >= pi if it covers all phi. */
static double disc_halfwidth(double tc, double R, double ta, double tb) {
  /* band outside the disc's colatitude range */
  if (tb < tc - R || ta > tc + R) return -1.0;
  /* a pole inside the disc and inside the band -> all longitudes */
  if (ta <= 0.0 && tc <= R) return 4.0 * OR_PI;
  if (tb >= OR_PI && tc + R >= OR_PI) return 4.0 * OR_PI;
  const double st = sin(tc), ct = cos(tc), cr = cos(R);
  if (st <= 0.0) return 4.0 * OR_PI;
  /* X(theta) = (cos R - cos tc cos theta) / (sin tc sin theta) has a single
   * minimum at cos theta = cos tc / cos R; the widest phi extent over the
   * band is acos of the smallest X there. */
  double lo = ta > tc - R ? ta : tc - R;
  double hi = tb < tc + R ? tb : tc + R;
  if (lo < 1e-300) lo = 1e-300;
  if (hi > OR_PI - 1e-16) hi = OR_PI - 1e-16;
  double tstar = (fabs(ct / cr) <= 1.0) ? acos(ct / cr) : lo;
  if (tstar < lo) tstar = lo;
  if (tstar > hi) tstar = hi;
  const double cand[3] = {lo, hi, tstar};
  double xmin = INFINITY;
  for (int i = 0; i < 3; ++i) {
    const double th = cand[i];
    const double x = (cr - ct * cos(th)) / (st * sin(th));
    if (x < xmin) xmin = x;
  }
  if (xmin <= -1.0) return 4.0 * OR_PI;
  if (xmin > 1.0) return -1.0;
  return acos(xmin);
}

/* Pixels of all rings whose box meets the disc; returns the count written
 * (or needed, when it exceeds cap). */
int64_t or_query_disc(int64_t ns, double lon_deg, double lat_deg, double radius_rad,
                      int64_t* out, int64_t cap) {
  const double tc = (90.0 - lat_deg) * OR_DEG2RAD;
  const double pc = or_lon_fold_deg(lon_deg) * OR_DEG2RAD;
  int64_t nout = 0;
  for (int64_t i = 1; i <= 4 * ns - 1; ++i) {
    const double ta = ring_theta(ns, i - 1), tb = ring_theta(ns, i + 1);
    const double hw = disc_halfwidth(tc, radius_rad, ta, tb);
    if (hw < 0.0) continue;
    int64_t count, first;
    double z, phase;
    or_ring_info(ns, i, &count, &first, &z, &phase);
    const double dphi = 2.0 * OR_PI / (double)count;
    const double W = hw + 0.5 * dphi + 1e-12;
    if (W >= OR_PI) {
      for (int64_t j = 0; j < count; ++j) {
        if (nout < cap) out[nout] = first + j;
        ++nout;
      }
      continue;
    }
    /* pixel centres (j + phase) * dphi within [pc - W, pc + W], modulo 2 pi */
    const int64_t jlo = (int64_t)ceil((pc - W) / dphi - phase);
    const int64_t jhi = (int64_t)floor((pc + W) / dphi - phase);
    for (int64_t jj = jlo; jj <= jhi; ++jj) {
      int64_t j = jj % count;
      if (j < 0) j += count;
      if (nout < cap) out[nout] = first + j;
      ++nout;
    }
  }
  return nout;
}

/* Eq. 4-5: the disc of ring i queried once at phi = 180 deg and moved along
 * the ring.  For every disc pixel p in ring r with n_r pixels and first index
 * s_r, the shift by dtheta gives p~ = s_r + ((p - s_r + dp) mod n_r) with
 * dp = round(dtheta n_r / (2 pi)).  The rounding of dp moves a pixel by at
 * most half a spacing, so the query radius must carry that slack for the
 * shifted disc to stay a superset. */
int64_t or_query_disc_shifted(int64_t ns, double lon_deg, double lat_deg, double radius_rad,
                              int64_t* out, int64_t cap) {
  /* the unshifted disc at phi = 180 deg, radius widened by the largest half
   * spacing any ring can have (pi / 4 for the 4-pixel ring) is far too wide;
   * instead widen per ring below by adding one pixel on each side. */
  int64_t base_cap = 1 << 16;
  int64_t* base = (int64_t*)malloc((size_t)base_cap * sizeof(int64_t));
  if (!base) return -1;
  int64_t nb = or_query_disc(ns, 180.0, lat_deg, radius_rad, base, base_cap);
  if (nb > base_cap) {
    free(base);
    base_cap = nb;
    base = (int64_t*)malloc((size_t)base_cap * sizeof(int64_t));
    if (!base) return -1;
    nb = or_query_disc(ns, 180.0, lat_deg, radius_rad, base, base_cap);
  }
  const double dtheta = (or_lon_fold_deg(lon_deg) - 180.0) * OR_DEG2RAD;
  int64_t nout = 0;
  for (int64_t q = 0; q < nb; ++q) {
    const int64_t p = base[q];
    const int64_t r = or_pix2ring(ns, p);
    int64_t count, first;
    double z, phase;
    or_ring_info(ns, r, &count, &first, &z, &phase);
    const int64_t dp = (int64_t)llround(dtheta * (double)count / (2.0 * OR_PI));
    for (int64_t e = -1; e <= 1; ++e) {      /* one pixel of rounding slack */
      int64_t j = (p - first + dp + e) % count;
      if (j < 0) j += count;
      if (nout < cap) out[nout] = first + j;
      ++nout;
    }
  }
  free(base);
  return nout;
}

/* ------------------------------------------------------------------------ */
/* Stable sort by key and CSR (replaces the paper's hash tables, Sect. 3.4)   */
/* ------------------------------------------------------------------------ */
static const int64_t* g_sort_keys;
static int cmp_key_then_index(const void* a, const void* b) {
  const int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  if (g_sort_keys[i] < g_sort_keys[j]) return -1;
  if (g_sort_keys[i] > g_sort_keys[j]) return 1;
  return (i < j) ? -1 : (i > j);
}

/* perm = indices ordered by (key, original index): a stable sort by key. */
void or_sort_stable(int64_t n, const int64_t* keys, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  g_sort_keys = keys;
  qsort(perm, (size_t)n, sizeof(int64_t), cmp_key_then_index);
}

/* Unique keys of a sorted key array with CSR offsets; returns U. */
int64_t or_csr(int64_t n, const int64_t* sorted_keys, int64_t* uniq, int64_t* off) {
  int64_t u = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (i == 0 || sorted_keys[i] != sorted_keys[i - 1]) {
      uniq[u] = sorted_keys[i];
      off[u] = i;
      ++u;
    }
  }
  off[u] = n;
  return u;
}

/* ring_off[i] = first sorted position whose pixel lies in ring >= i, for
 * i = 0 .. 4ns (ring 0 and ring 4ns are sentinels). */
void or_ring_offsets(int64_t ns, int64_t n, const int64_t* sorted_keys, int64_t* ring_off) {
  int64_t pos = 0;
  for (int64_t i = 0; i <= 4 * ns; ++i) {
    while (pos < n && or_pix2ring(ns, sorted_keys[pos]) < i) ++pos;
    ring_off[i] = pos;
  }
}

/* ------------------------------------------------------------------------ */
/* HEALPix lookup gridder (Sect. 2.2 steps 1-3c, Sect. 3.4)                  */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t h; int64_t t; } hp_entry;
static int cmp_i64(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x < y) ? -1 : (x > y);
}
static int cmp_entry(const void* a, const void* b) {
  const hp_entry* x = (const hp_entry*)a;
  const hp_entry* y = (const hp_entry*)b;
  if (x->h != y->h) return (x->h < y->h) ? -1 : 1;
  return (x->t < y->t) ? -1 : (x->t > y->t);
}

/* mode 0: disc around each sample's own position;
 * mode 1: per-ring disc moved along the ring (Eq. 4-5).
 * The exact cut d <= r is applied to every candidate, so both modes give the
 * Eq. 1-3 result of the brute-force gridder. */
int or_grid_lookup(int64_t ns, int32_t mode, int64_t P, const double* lon_t,
                   const double* lat_t, int64_t N, const double* lon_s, const double* lat_s,
                   int32_t C, const double* data, const double* omega, const or_kernel* k,
                   double* num, double* wsum, double* out, double* sabs, int64_t* npairs) {
  /* step 1-2: HEALPix index of every target, organised as a lookup table */
  hp_entry* tab = (hp_entry*)malloc((size_t)(P > 0 ? P : 1) * sizeof(hp_entry));
  or_acc* anum = (or_acc*)calloc((size_t)(P * C > 0 ? P * C : 1), sizeof(or_acc));
  or_acc* aabs = (or_acc*)calloc((size_t)(P * C > 0 ? P * C : 1), sizeof(or_acc));
  or_acc* aw = (or_acc*)calloc((size_t)(P > 0 ? P : 1), sizeof(or_acc));
  int64_t cap = 1 << 16;
  int64_t* disc = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
  if (!tab || !anum || !aabs || !aw || !disc) {
    free(tab); free(anum); free(aabs); free(aw); free(disc);
    return 1;
  }
  for (int64_t t = 0; t < P; ++t) {
    tab[t].h = or_ang2pix_ring(ns, lon_t[t], lat_t[t]);
    tab[t].t = t;
  }
  qsort(tab, (size_t)P, sizeof(hp_entry), cmp_entry);
  const double r = k->support_deg * OR_DEG2RAD;
  int64_t pairs = 0;
  /* step 3: every sample queries its disc and is matched against the table */
  for (int64_t n = 0; n < N; ++n) {
    int64_t nd;
    for (;;) {
      nd = (mode == 1) ? or_query_disc_shifted(ns, lon_s[n], lat_s[n], r, disc, cap)
                       : or_query_disc(ns, lon_s[n], lat_s[n], r, disc, cap);
      if (nd < 0) { nd = 0; break; }
      if (nd <= cap) break;
      free(disc);
      cap = nd;
      disc = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
      if (!disc) { free(tab); free(anum); free(aabs); free(aw); return 1; }
    }
    /* a shifted disc may list a pixel twice: sort and skip duplicates */
    if (mode == 1) qsort(disc, (size_t)nd, sizeof(int64_t), cmp_i64);
    for (int64_t q = 0; q < nd; ++q) {
      if (mode == 1 && q > 0 && disc[q] == disc[q - 1]) continue;
      const int64_t h = disc[q];
      /* binary search for the first table entry with key h */
      int64_t lo = 0, hi = P;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (tab[mid].h < h) lo = mid + 1; else hi = mid;
      }
      for (int64_t e = lo; e < P && tab[e].h == h; ++e) {
        const int64_t t = tab[e].t;
        int inside;
        double d;
        const double w = kernel_eval(k, lon_t[t], lat_t[t], lon_s[n], lat_s[n], &inside, &d);
        if (!inside) continue;
        ++pairs;
        const double ww = w * (omega ? omega[n] : 1.0);
        acc_add(&aw[t], ww);
        for (int32_t c = 0; c < C; ++c) {
          acc_add(&anum[t * C + c], ww * data[n * C + c]);
          acc_add(&aabs[t * C + c], fabs(ww * data[n * C + c]));
        }
      }
    }
  }
  (void)r;
  finish_maps(P, C, anum, aw, aabs, num, wsum, out, sabs);
  if (npairs) *npairs = pairs;
  free(tab); free(anum); free(aabs); free(aw); free(disc);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (degridding) and kernel-width derivative                          */
/* ------------------------------------------------------------------------ */
/* The normalised gridding of Eq. 3 is linear in the data: R = G D with
 * G[p][n] = omega_n w_pn / W_p (rows with W_p = 0 are zero).  The adjoint
 * applies the transpose: xhat[n][c] = sum_p G[p][n] y[p][c]. */
int or_degrid_bruteforce(int64_t P, const double* lon_t, const double* lat_t, int64_t N,
                         const double* lon_s, const double* lat_s, int32_t C,
                         const double* omega, const or_kernel* k, const double* y,
                         double* xhat) {
  or_acc* aw = (or_acc*)calloc((size_t)(P > 0 ? P : 1), sizeof(or_acc));
  or_acc* ax = (or_acc*)calloc((size_t)(N * C > 0 ? N * C : 1), sizeof(or_acc));
  if (!aw || !ax) { free(aw); free(ax); return 1; }
  for (int64_t p = 0; p < P; ++p)
    for (int64_t n = 0; n < N; ++n) {
      int inside;
      double d;
      const double w = kernel_eval(k, lon_t[p], lat_t[p], lon_s[n], lat_s[n], &inside, &d);
      if (inside) acc_add(&aw[p], w * (omega ? omega[n] : 1.0));
    }
  for (int64_t p = 0; p < P; ++p) {
    const double W = acc_get(&aw[p]);
    if (!(W > 0.0)) continue;
    for (int64_t n = 0; n < N; ++n) {
      int inside;
      double d;
      const double w = kernel_eval(k, lon_t[p], lat_t[p], lon_s[n], lat_s[n], &inside, &d);
      if (!inside) continue;
      const double g = w * (omega ? omega[n] : 1.0) / W;
      for (int32_t c = 0; c < C; ++c) acc_add(&ax[n * C + c], g * y[p * C + c]);
    }
  }
  for (int64_t i = 0; i < N * C; ++i) xhat[i] = acc_get(&ax[i]);
  free(aw); free(ax);
  return 0;
}

/* Normalised interpolation (map -> samples; the degridding reading in which
 * each sample gets the kernel-weighted mean of the map around it, the mirror
 * of Eq. 1-3): xhat[n][c] = sum_p w_pn y[p][c] / V_n, V_n = sum_p w_pn over
 * the targets with d_pn <= r; NaN where V_n = 0.  Sample weights do not
 * enter.  vsum[n] = V_n (may be NULL). */
int or_interp_bruteforce(int64_t P, const double* lon_t, const double* lat_t, int64_t N,
                         const double* lon_s, const double* lat_s, int32_t C,
                         const or_kernel* k, const double* y, double* xhat, double* vsum) {
  or_acc* ax = (or_acc*)calloc((size_t)(C > 0 ? C : 1), sizeof(or_acc));
  if (!ax) return 1;
  for (int64_t n = 0; n < N; ++n) {
    or_acc av = {0.0, 0.0};
    for (int32_t c = 0; c < C; ++c) ax[c] = av;
    for (int64_t p = 0; p < P; ++p) {
      int inside;
      double d;
      const double w = kernel_eval(k, lon_t[p], lat_t[p], lon_s[n], lat_s[n], &inside, &d);
      if (!inside) continue;
      acc_add(&av, w);
      for (int32_t c = 0; c < C; ++c) acc_add(&ax[c], w * y[p * C + c]);
    }
    const double V = acc_get(&av);
    for (int32_t c = 0; c < C; ++c) xhat[n * C + c] = (V > 0.0) ? acc_get(&ax[c]) / V : NAN;
    if (vsum) vsum[n] = V;
  }
  free(ax);
  return 0;
}

/* d R_pc / d sigma for the circular Gaussian with the support r held fixed:
 * w' = dw/dsigma = w d^2 / sigma^3 (d and sigma in degrees), and
 * dR/dsigma = (sum_n omega w' D - R sum_n omega w') / W. */
int or_dsigma_bruteforce(int64_t P, const double* lon_t, const double* lat_t, int64_t N,
                         const double* lon_s, const double* lat_s, int32_t C,
                         const double* data, const double* omega, const or_kernel* k,
                         double* dR) {
  or_acc* aw = (or_acc*)calloc((size_t)(P > 0 ? P : 1), sizeof(or_acc));
  or_acc* awp = (or_acc*)calloc((size_t)(P > 0 ? P : 1), sizeof(or_acc));
  or_acc* an = (or_acc*)calloc((size_t)(P * C > 0 ? P * C : 1), sizeof(or_acc));
  or_acc* anp = (or_acc*)calloc((size_t)(P * C > 0 ? P * C : 1), sizeof(or_acc));
  if (!aw || !awp || !an || !anp) { free(aw); free(awp); free(an); free(anp); return 1; }
  const double s = k->sigma_deg;
  for (int64_t p = 0; p < P; ++p)
    for (int64_t n = 0; n < N; ++n) {
      int inside;
      double d;
      const double w = kernel_eval(k, lon_t[p], lat_t[p], lon_s[n], lat_s[n], &inside, &d);
      if (!inside) continue;
      const double om = omega ? omega[n] : 1.0;
      const double dd = d / OR_DEG2RAD;
      const double wp = w * dd * dd / (s * s * s);
      acc_add(&aw[p], om * w);
      acc_add(&awp[p], om * wp);
      for (int32_t c = 0; c < C; ++c) {
        acc_add(&an[p * C + c], om * w * data[n * C + c]);
        acc_add(&anp[p * C + c], om * wp * data[n * C + c]);
      }
    }
  for (int64_t p = 0; p < P; ++p) {
    const double W = acc_get(&aw[p]), Wp = acc_get(&awp[p]);
    for (int32_t c = 0; c < C; ++c) {
      if (!(W > 0.0)) { dR[p * C + c] = NAN; continue; }
      const double R = acc_get(&an[p * C + c]) / W;
      dR[p * C + c] = (acc_get(&anp[p * C + c]) - R * Wp) / W;
    }
  }
  free(aw); free(awp); free(an); free(anp);
  return 0;
}
