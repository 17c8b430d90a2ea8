/*
 * FP64 fmod and remainder of the oracle (exact results; u35 = u10).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * fmod follows Section 5.9 (Algorithm 1, long division with floating-point
 * "digits": r_{k+1} = r_k - q_k d for any integer q_k in [(r_k/d)/2, r_k/d])
 * and the Appendix B listing: one reciprocal (reading R33, oracle_fmod_recip),
 * q = trunc(nextafter(r, 0) * rd), the fix-ups for 1 < r/d < 3 and r == d, r kept exact in
 * DD, the 2^54 rescale of subnormal divisors.  The listing is valid only for
 * x/y < DBL_MAX with at most 21 iterations; here (reading A8) each iteration
 * divides by D = d 2^j with j = max(kmin, ilogb(r) - ilogb(d) - 1000), so r/D
 * stays below 2^1001 (j = 0, i.e. the listing itself, whenever n/d < 2^1000);
 * a subnormal divisor (kmin = 54) first reduces r below d 2^54 and then runs
 * the listing's rescaled loop.  Iterations: ceil(log2(n/d) / 52) (Appendix C)
 * plus the fix-up steps, at most 44 for any pair of doubles.
 *
 * remainder (reading A9): r2 = fmod(|x|, 2|y|) (|x| itself when 2|y|
 * overflows), then subtract |y| once or twice by comparing 2 r2 with |y|
 * (ties to the even quotient); every subtraction is exact (Sterbenz).
 */
#include "common.h"

#define FMOD_MAXIT 48

static double rdown(double v) { return nextafter(v, 0.0); }
static double dfrom(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static float ffrom(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

/* The reciprocal of the divisor (reading R33): Section 5.9 lets q_k be any
 * integer in [(r_k/d)/2, r_k/d] and says the division need not be correctly
 * rounded; the listing's nextafter(1/d, 0) is one such choice.  Here: the
 * binary32 reciprocal of d's significand m (truncated to 24 bits), widened
 * exactly, two Newton steps y += y (1 - m y) with fma, then two units in the
 * last place down, scaled by 2^-ilogb(d) through the exponent field.  The
 * result never exceeds 1/d and is within 2^-50 of it (pinned with exact
 * rationals), which keeps the proof's factor u above 5/6.  For d >= 2^1021,
 * where 1/d approaches the subnormal range, the listing's form is kept. */
double oracle_fmod_recip(double d) {
  uint64_t b = dbits(d);
  int e = (int)(b >> 52) - 1023;
  if (e >= 1021) return rdown(1.0 / d);
  uint64_t man = b & 0x000FFFFFFFFFFFFFULL;
  double m = dfrom(0x3FF0000000000000ULL | man);
  float mf = ffrom(0x3F800000U | (uint32_t)(man >> 29));      /* m truncated to 24 bits */
  float rf = 1.0f / mf;                                       /* in (1/2, 1] */
  uint32_t rb = fbits(rf);
  double y = dfrom(((uint64_t)((rb >> 23) + 896) << 52) | ((uint64_t)(rb & 0x7FFFFF) << 29));  /* exact */
  double t = fma(-m, y, 1.0);
  y = fma(y, t, y);
  t = fma(-m, y, 1.0);
  y = fma(y, t, y);
  y = dfrom(dbits(y) - 2);                                    /* two ulps down: y < 1/m */
  return dfrom(dbits(y) - ((uint64_t)(int64_t)e << 52));      /* y 2^-e, normal */
}

/* one step of Algorithm 1 with divisor D and rD = nextafter(1/D, 0) */
static dd_t fmod_step(dd_t r, double D, double rD) {
  double q = trunc(rdown(r.x) * rD);
  q = (3 * D > r.x && r.x > D) ? 2 : q;
  q = (2 * D > r.x && r.x > D) ? 1 : q;
  q = r.x == D ? (r.y >= 0 ? 1 : 0) : q;
  return ddnormalize_d2_d2(ddadd2_d2_d2_d2(r, ddmul_d2_d_d(q, -D)));
}

/* |x| mod |y| for finite x and finite non-zero y; *iters counts steps */
static double fmod_abs(double n, double d, int *iters) {
  int sub = d < 0x1p-1022;
  int kmin = sub ? 54 : 0;
  double dmin = ldexp(d, kmin);
  double rd0 = oracle_fmod_recip(dmin);
  int ed = ilogb(d);
  dd_t r = dd(n, 0);
  int it = 0;
  for (; it < FMOD_MAXIT && r.x >= dmin; it++) {
    int j = ilogb(r.x) - ed - 1000;
    if (j < kmin) j = kmin;
    r = fmod_step(r, ldexp(d, j), ldexp(rd0, kmin - j));
  }
  double ret;
  if (sub) {                      /* the listing's rescaled loop, r < d 2^54 now */
    r = dd(r.x * 0x1p54, r.y * 0x1p54);
    for (int k = 0; k < 4 && r.x >= dmin; k++, it++) r = fmod_step(r, dmin, rd0);
    ret = r.x * 0x1p-54;
    if (r.x + r.y == dmin) ret = 0;
  } else {
    ret = r.x;
    if (r.x + r.y == d) ret = 0;
  }
  *iters = it;
  return ret;
}

double oracle_fmod_u10_f64(double x, double y) {
  double n = fabs(x), d = fabs(y);
  int ok = isfinite(n) && d > 0 && isfinite(d);
  int it;
  double ret = fmod_abs(ok ? n : 0.0, ok ? d : 1.0, &it);
  ret = copysign(ret, x);
  if (n < d) ret = x;            /* includes finite x with infinite y */
  if (!(d > 0) || isinf(n) || isnan(x) || isnan(y)) ret = NAN;
  return canon(ret);
}
double oracle_fmod_u35_f64(double x, double y) { return oracle_fmod_u10_f64(x, y); }

/* iteration count of the fmod loop (for the trip-count pin) */
int oracle_fmod_iters(double x, double y) {
  double n = fabs(x), d = fabs(y);
  if (!(isfinite(n) && d > 0 && isfinite(d))) return 0;
  int it;
  fmod_abs(n, d, &it);
  return it;
}

double oracle_remainder_u10_f64(double x, double y) {
  double n = fabs(x), d = fabs(y);
  int ok = isfinite(n) && d > 0 && isfinite(d);
  double nn = ok ? n : 0.0, dd2 = ok ? d : 1.0;
  double r2 = nn;
  int it;
  if (dd2 <= 0x1.fffffffffffffp1022) r2 = fmod_abs(nn, 2 * dd2, &it);   /* 2|y| finite */
  if (r2 + r2 > dd2) {            /* quotient 1, or 2 when r2 >= 3|y|/2 */
    r2 = r2 - dd2;
    if (r2 + r2 >= dd2) r2 = r2 - dd2;
  }
  double ret = signbit(x) ? -r2 : r2;
  if (isinf(y) && isfinite(x)) ret = x;
  if (!(d > 0) || isinf(n) || isnan(x) || isnan(y)) ret = NAN;
  return canon(ret);
}
double oracle_remainder_u35_f64(double x, double y) { return oracle_remainder_u10_f64(x, y); }

/* the quotients q_k and partial remainders r_k (heads) of fmod's loop, for
 * the worked example of Section 5.9; returns the number of steps */
int oracle_fmod_trace(double x, double y, double *qs, double *rs, int maxk) {
  double n = fabs(x), d = fabs(y);
  if (!(isfinite(n) && d >= 0x1p-1022 && isfinite(d))) return 0;
  double rd0 = oracle_fmod_recip(d);
  int ed = ilogb(d), k = 0;
  dd_t r = dd(n, 0);
  while (k < maxk && k < FMOD_MAXIT && r.x >= d) {
    int j = ilogb(r.x) - ed - 1000;
    if (j < 0) j = 0;
    double D = ldexp(d, j), rD = ldexp(rd0, -j);
    double q = trunc(rdown(r.x) * rD);
    q = (3 * D > r.x && r.x > D) ? 2 : q;
    q = (2 * D > r.x && r.x > D) ? 1 : q;
    q = r.x == D ? (r.y >= 0 ? 1 : 0) : q;
    r = ddnormalize_d2_d2(ddadd2_d2_d2_d2(r, ddmul_d2_d_d(q, -D)));
    qs[k] = q;
    rs[k] = r.x;
    k++;
  }
  return k;
}
