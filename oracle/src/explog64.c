/*
 * FP64 exp, log and pow of the oracle, 1-ULP (u10) and 3.5-ULP (u35).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * exp (Section 5.6): x = k ln2 + r with |r| <= ln2/2 by a two-constant
 *   Cody-Waite step, e^r by one polynomial without DD, then 2^k added in two
 *   multiplications so that results near overflow and in the subnormal range
 *   are rounded once.
 * log (Section 5.5): arguments below DBL_MIN are scaled by 2^64;
 *   e = floor(log2(4a/3)) and m = a 2^-e in [0.75, 1.5) (taken exactly from
 *   the significand); log m = z + z^3 P(z^2) with z = 2(m-1)/(m+1) in DD;
 *   log a = e ln2 + log m.
 * pow (Section 5.7): e^(y log|x|) with the logarithm and the product in DD,
 *   an 11-term internal log and a 13-term internal exp; the C99 Annex F
 *   special cases are selected at the end (Section 5.10).
 */
#include "common.h"
#include "coeffs64.h"
#include "explog64.h"

#define R_LN2 0x1.71547652b82fep0    /* RN(1/ln2) */
#define L2A 0x1.62e42fefa39efp-1     /* RN(ln2) */
#define L2B 0x1.abc9e3b39803fp-56    /* RN(ln2 - L2A) */
#define L2H 0x1.62e42fefa3800p-1     /* ln2 to 42 bits: e*L2H is exact for |e| < 2^11 */
#define L2L 0x1.ef35793c76730p-45    /* RN(ln2 - L2H) */

/* y * 2^k in two steps, y * 2^k1 then * 2^k2 with both factors normal
 * powers of two, so that the result is rounded once even when it is
 * subnormal; each step is an exponent operation (ldexp, correctly rounded) */
static double scale2(double y, int k) {
  int k1 = k / 2, k2 = k - k1;
  return ldexp(ldexp(y, k1), k2);
}
double oracle_scale2(double y, int k) { return scale2(y, k); }

/* ---------------- exp ---------------- */
static const double EXP_U10[11] = { EXP_U10_COEFFS };
static const double EXP_U35[9] = { EXP_U35_COEFFS };

/* u35: e^r = 1 + (r + r^2 u(r)) in double, r rounded once */
static double exp_core(double x, const double *c, int nc) {
  double xc = fabs(x) <= 746 ? x : 0.0;   /* keeps k small; out-of-range is selected below */
  double k = rint(xc * R_LN2);
  double r = fma(k, -L2A, xc);
  r = fma(k, -L2B, r);
  double s = r * r;
  double u = poly_d(r, c, nc);
  double v = fma(s, u, r);
  double y = scale2(1.0 + v, (int)k);
  if (!(fabs(x) <= 746)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}

/* u10: the same reduction keeps the rounding residual rl of r = h - k L2B
 * (h = x - k L2A exact) and forms 1 + r as a DD, so that the only rounding
 * of order one ulp is the final one */
double oracle_exp_tail_u10(double r, double rl, double k) {
  double s = r * r;
  double w = fma(s, poly_d(r, EXP_U10, 11), rl);
  dd_t o = ddadd_d2_d_d(1.0, r);
  return scale2(o.x + (o.y + w), (int)k);
}

static double exp_core_u10(double x) {
  double xc = fabs(x) <= 746 ? x : 0.0;
  double k = rint(xc * R_LN2);
  double h = fma(k, -L2A, xc);
  double r = fma(k, -L2B, h);
  double rl = fma(k, -L2B, h - r);
  double y = oracle_exp_tail_u10(r, rl, k);
  if (!(fabs(x) <= 746)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}
double oracle_exp_u10_f64(double x) { return exp_core_u10(x); }
double oracle_exp_u35_f64(double x) { return exp_core(x, EXP_U35, 9); }

/* ---------------- log ---------------- */
static const double LOG_U10[8] = { LOG_U10_COEFFS };
static const double LOG_U35[7] = { LOG_U35_COEFFS };

/* a > 0 finite: a = m 2^e, m in [0.75, 1.5) (Section 5.5 with the 2^64
 * rescale of subnormals) */
static double log_reduce(double a, int *e) {
  int off = 0;
  if (a < 0x1p-1022) { a *= 0x1p64; off = 64; }
  int ex = ilogb(a);
  double m = ldexp(a, -ex);
  if (m >= 1.5) { m *= 0.5; ex++; }
  *e = ex - off;
  return m;
}

static double log_special(double x, double y) {
  if (x == 0) return -INFINITY;
  if (x < 0 || isnan(x)) return NAN;
  if (isinf(x)) return INFINITY;
  return y;
}

double oracle_log_u10_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  double m = log_reduce(a, &e);
  dd_t den = ddadd_d2_d_d(1.0, m);
  dd_t z = dddiv_d2_d2_d2(dd(2.0 * (m - 1.0), 0), den);
  double t = z.x * z.x;
  double corr = (z.x * t) * poly_d(t, LOG_U10, 8);
  double ed = (double)e;
  dd_t r = ddadd_d2_d2_d2(dd(ed * L2H, ed * L2L), z);
  r = ddadd_d2_d2_d(r, corr);
  return canon(log_special(x, r.x + r.y));
}

double oracle_log_u35_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  double m = log_reduce(a, &e);
  double z = (2.0 * (m - 1.0)) * (1.0 / (1.0 + m));
  double t = z * z;
  double lm = fma(z * t, poly_d(t, LOG_U35, 7), z);
  double y = fma((double)e, L2A, lm);
  return canon(log_special(x, y));
}

/* log of a DD a > 0 with a normal, finite head: a = m 2^e, m in [0.75, 1.5)
 * (heads below DBL_MIN are scaled by 2^64 first); returns log m = z +
 * z^3 P(z^2) as a DD, with z = 2(m-1)/(m+1) in DD and the u10 polynomial,
 * and e through *ep (Section 5.5 applied to a DD argument). */
dd_t oracle_logm_u10(dd_t a, int *ep) {
  int off = 0;
  if (a.x < 0x1p-1022) { a = ddscale_d2_d2_d(a, 0x1p64); off = 64; }
  int ex = ilogb(a.x);
  dd_t m = ddscale_d2_d2_d(a, ldexp(1.0, -ex));
  if (m.x >= 1.5) { m = ddscale_d2_d2_d(m, 0.5); ex++; }
  dd_t num = ddscale_d2_d2_d(ddadd2_d2_d_d(m.x - 1.0, m.y), 2.0);
  dd_t den = ddadd2_d2_d_d2(1.0, m);
  dd_t z = dddiv_d2_d2_d2(num, den);
  double t = z.x * z.x;
  double corr = (z.x * t) * poly_d(t, LOG_U10, 8);
  *ep = ex - off;
  return ddadd_d2_d2_d(z, corr);
}

/* log m in double for the u35 forms: a = m 2^e as above, z rounded once
 * from the DD numerator */
double oracle_logm_u35(dd_t a, int *ep) {
  int off = 0;
  if (a.x < 0x1p-1022) { a = ddscale_d2_d2_d(a, 0x1p64); off = 64; }
  int ex = ilogb(a.x);
  dd_t m = ddscale_d2_d2_d(a, ldexp(1.0, -ex));
  if (m.x >= 1.5) { m = ddscale_d2_d2_d(m, 0.5); ex++; }
  double num = 2.0 * ((m.x - 1.0) + m.y);
  double z = num * (1.0 / (1.0 + m.x));
  double t = z * z;
  *ep = ex - off;
  return fma(z * t, poly_d(t, LOG_U35, 7), z);
}

/* log m in double with z = 2(m-1)/(m+1) corrected once: the reciprocal
 * quotient's residual num - z (1 + m) taken by fma (with the DD tail of m)
 * and added back through the reciprocal, then the 3.5-ULP polynomial; for
 * the 3.5-ULP forms whose logarithm is small against its argument's
 * rounding (asinh, acosh, atanh near 0 and 1) */
double oracle_logm_u20(dd_t a, int *ep) {
  int off = 0;
  if (a.x < 0x1p-1022) { a = ddscale_d2_d2_d(a, 0x1p64); off = 64; }
  int ex = ilogb(a.x);
  dd_t m = ddscale_d2_d2_d(a, ldexp(1.0, -ex));
  if (m.x >= 1.5) { m = ddscale_d2_d2_d(m, 0.5); ex++; }
  double num = 2.0 * ((m.x - 1.0) + m.y);
  double den = 1.0 + m.x;
  double rd = 1.0 / den;
  double z = num * rd;
  double r = fma(-z, den, num) - z * (((1.0 - den) + m.x) + m.y);   /* num - z (1 + m), the rounding of den included */
  z = fma(r, rd, z);
  double t = z * z;
  *ep = ex - off;
  return fma(z * t, poly_d(t, LOG_U35, 7), z);
}

/* ---------------- pow ---------------- */
static const double PL_C1H = POWLOG_C1H, PL_C1L = POWLOG_C1L;
static const double POWLOG[9] = { POWLOG_COEFFS };
static const double POWEXP[10] = { POWEXP_COEFFS };

/* log a in DD for finite a > 0 (11-term polynomial) */
static dd_t logk(double a) {
  int e;
  double m = log_reduce(a, &e);
  dd_t den = ddadd_d2_d_d(1.0, m);
  dd_t z = dddiv_d2_d2_d2(dd(2.0 * (m - 1.0), 0), den);
  dd_t t = ddsqu_d2_d2(z);
  double q = poly_d(t.x, POWLOG, 9);
  dd_t w = ddadd_d2_d2_d(dd(PL_C1H, PL_C1L), t.x * q);
  w = ddmul_d2_d2_d2(t, w);
  w = ddmul_d2_d2_d2(z, w);
  dd_t lm = ddadd_d2_d2_d2(z, w);
  double ed = (double)e;
  return ddadd_d2_d2_d2(dd(ed * L2H, ed * L2L), lm);
}

/* e^Y for a DD argument (13-term polynomial, the leading terms in DD) */
/* For |Y.x| <= 746: k = rint(Y.x / ln2) and e^(Y - k ln2) - 1 as a DD.
 * Y.x - k L2A is exact (k has at most 11 bits and |result| < 1/2), so the
 * reduced argument is a DD to about 2^-100. */
dd_t oracle_expk_s(dd_t Y, double *kp) {
  double k = rint(Y.x * R_LN2);
  double u = fma(k, -L2A, Y.x);
  dd_t r = ddadd2_d2_d_d(u, fma(k, -L2B, Y.y));
  dd_t q = ddscale_d2_d2_d(ddsqu_d2_d2(r), 0.5);
  double p = poly_d(r.x, POWEXP, 10);
  double v = ((r.x * r.x) * r.x) * p;
  dd_t s = ddadd2_d2_d2_d2(r, q);
  s = ddadd2_d2_d2_d(s, v);
  *kp = k;
  return s;
}

static double expk(dd_t Y) {
  double yh = Y.x, yl = Y.y;
  if (!(fabs(yh) <= 746)) { yh = 0; yl = 0; }
  double k;
  dd_t s = oracle_expk_s(dd(yh, yl), &k);
  s = ddadd_d2_d_d2(1.0, s);
  double y = scale2(s.x + s.y, (int)k);
  if (!(fabs(Y.x) <= 746)) y = Y.x > 0 ? INFINITY : 0.0;
  return y;
}

/* log of a DD y > 0 (finite) with the internal log of pow: y = m 2^e with m
 * in [0.75, 1.5) taken from the head, z = 2(m-1)/(m+1) in DD and the 11-term
 * DD polynomial; about 2^-66 relative */
dd_t oracle_logk_dd(dd_t y) {
  int off = 0;
  if (y.x < 0x1p-1022) { y = ddscale_d2_d2_d(y, 0x1p64); off = 64; }
  int ex = ilogb(y.x);
  dd_t m = ddscale_d2_d2_d(y, ldexp(1.0, -ex));
  if (m.x >= 1.5) { m = ddscale_d2_d2_d(m, 0.5); ex++; }
  dd_t num = ddscale_d2_d2_d(ddadd2_d2_d_d(m.x - 1.0, m.y), 2.0);
  dd_t z = dddiv_d2_d2_d2(num, ddadd2_d2_d_d2(1.0, m));
  dd_t t = ddsqu_d2_d2(z);
  double q = poly_d(t.x, POWLOG, 9);
  dd_t w = ddadd_d2_d2_d(dd(PL_C1H, PL_C1L), t.x * q);
  w = ddmul_d2_d2_d2(t, w);
  w = ddmul_d2_d2_d2(z, w);
  dd_t lm = ddadd_d2_d2_d2(z, w);
  double ed = (double)(ex - off);
  return ddadd2_d2_d2_d2(dd(ed * L2H, ed * L2L), lm);
}

/* e^Y for a DD Y (the internal exp of pow): overflow to +inf, underflow with
 * subnormals rounded once */
double oracle_exp_dd(dd_t Y) { return expk(Y); }

double oracle_pow_u10_f64(double x, double y) {
  double ax = fabs(x);
  double axc = (ax > 0 && ax <= 0x1.fffffffffffffp1023) ? ax : 1.0;
  double yc = isfinite(y) ? y : 0.0;
  int yint = isfinite(y) && y == trunc(y);
  int yodd = yint && fabs(y) < 0x1p53 && ((int64_t)y & 1);
  double r = expk(ddmul_d2_d2_d(logk(axc), yc));
  if (x < 0 && yodd) r = -r;
  if (x < 0 && isfinite(x) && isfinite(y) && !yint) r = NAN;
  if (x == 0) {
    if (y < 0) r = yodd ? copysign(INFINITY, x) : INFINITY;
    else if (y > 0) r = yodd ? x : 0.0;
  }
  if (isinf(y)) {
    if (ax == 1) r = 1.0;
    else r = ((ax < 1) == (y < 0)) ? INFINITY : 0.0;
  }
  if (isinf(x)) {
    if (x > 0) r = y < 0 ? 0.0 : INFINITY;
    else if (y < 0) r = yodd ? -0.0 : 0.0;
    else r = yodd ? -INFINITY : INFINITY;
  }
  if (isnan(x) || isnan(y)) r = NAN;
  if (y == 0 || x == 1) r = 1.0;
  return canon(r);
}

/* The DD internals leave nothing a shorter polynomial could save within the
 * 3.5-ULP bound at |y log x| ~ 700, so the u35 entry point is the u10
 * algorithm. */
double oracle_pow_u35_f64(double x, double y) { return oracle_pow_u10_f64(x, y); }
