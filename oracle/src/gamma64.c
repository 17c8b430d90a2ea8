/*
 * FP64 tgamma and lgamma of the oracle (u10; the u35 entry points run the
 * same algorithms).  The paper lists them in the library without their
 * steps; this is the design used here.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#include "common.h"
#include "coeffs64.h"
#include "explog64.h"

/* ---------------- tgamma, lgamma ----------------
 * For y > 0 given as a DD:
 *   y >= 8         Stirling: (y - 1/2) log y - y + log(2 pi)/2 + G(1/y^2)/y,
 *                  the logarithm the 11-term DD one of pow (Section 5.7)
 *   1.75 <= y < 2.5  lgamma(2 + e) = e (c1 + e (c2 + e Q(e))), e = y - 2,
 *                  relative accuracy across the zero at 2
 *   1.25 <= y < 1.75 lgamma(1.5 + u) = c0 + u (c1 + u (c2 + u Q(u))) around the minimum
 *   0.5 <= y < 1.25  lgamma(y + 1) - log y with those polynomials (the
 *                  zero at 1 cancels only by a factor of about two)
 *   otherwise      lgamma(y + n) - log(y (y+1) ... (y+n-1)) with y + n in
 *                  [8, 9), the product in DD
 * y < 0 (not an integer): reflection, lgamma(y) = log pi - log|sin(pi y)| -
 * lgamma(1 - y), sin(pi y) from y reduced exactly to [-1/2, 1/2] and an odd
 * polynomial with DD leading terms.  tgamma(y) = exp(L) with L the DD
 * log-gamma for y > 0 (so only its absolute error matters); for y < 0 the
 * reflection in linear form, pi / (sin(pi y) e^g) with g = lgamma(1 - y)
 * (one DD logarithm fewer than through L).  Near the zeros of lgamma on the negative axis the reflection
 * cancels, as in every libm: the relative error there is reported
 * separately (absolute error bound).  Both u35 entry points run the u10
 * algorithm. */
#define LOG2PI_H 0x1.d67f1c864beb5p-1   /* log(2 pi)/2 as a DD */
#define LOG2PI_L -0x1.65b5a1b7ff5dfp-55
#define LOGPI_H 0x1.250d048e7a1bdp+0     /* log(pi) as a DD */
#define LOGPI_L 0x1.7abf2ad8d5088p-57
#define PI_H 0x1.921fb54442d18p+1
#define PI_L 0x1.1a62633145c07p-53
/* 200 ln 2 as a DD: 200 times the 42-bit head of ln 2 (exact) and RN(200 times its tail) */
#define LN2X200_H 0x1.1542457337bc0p+7
#define LN2X200_L 0x1.82e1c6b73c89ep-37

static const double LG_RH[4] = { LGAMMA_R2_HEAD };
static const double LG_RP[16] = { LGAMMA_R2_COEFFS };
static const double LG_MH[6] = { LGAMMA_M_HEAD };
static const double LG_MP[15] = { LGAMMA_M_COEFFS };
static const double LG_ST[10] = { LGAMMA_ST_COEFFS };
static const double SP_H[2] = { SINPI_HEAD };
static const double SP_P[11] = { SINPI_COEFFS };

/* lgamma(2 + e) as a DD for -0.25 <= e < 0.5 */
static dd_t lg_r2(dd_t e) {
  double p = poly_d(e.x, LG_RP, 16);
  dd_t in = ddadd2_d2_d2_d(dd(LG_RH[2], LG_RH[3]), e.x * p);
  in = ddadd2_d2_d2_d2(dd(LG_RH[0], LG_RH[1]), ddmul_d2_d2_d2(in, e));
  return ddmul_d2_d2_d2(in, e);
}

/* lgamma(1.5 + u) as a DD for -0.25 <= u < 0.25 */
static dd_t lg_m(dd_t u) {
  double p = poly_d(u.x, LG_MP, 15);
  dd_t in = ddadd2_d2_d2_d(dd(LG_MH[4], LG_MH[5]), u.x * p);
  in = ddadd2_d2_d2_d2(dd(LG_MH[2], LG_MH[3]), ddmul_d2_d2_d2(in, u));
  return ddadd2_d2_d2_d2(dd(LG_MH[0], LG_MH[1]), ddmul_d2_d2_d2(in, u));
}

/* Stirling's form for a DD y >= 8 */
static dd_t lg_stirling(dd_t y) {
  dd_t ly = oracle_logk_dd(y);
  dd_t r = ddmul_d2_d2_d2(ddadd2_d2_d2_d(y, -0.5), ly);
  r = ddadd2_d2_d2_d2(r, dd(-y.x, -y.y));
  /* from 2^60 on, log(2 pi)/2 + G(1/y^2)/y < 0.92 is under 2^-12 ulp of
   * (y - 1/2) log y - y (ulp >= 2^13) and is left out */
  if (y.x >= 0x1p60) return r;
  r = ddadd2_d2_d2_d2(r, dd(LOG2PI_H, LOG2PI_L));
  double ry = 1.0 / y.x;                      /* one reciprocal gives w = 1/y^2 and G(w)/y */
  double w = ry * ry;
  return ddadd2_d2_d2_d(r, poly_d(w, LG_ST, 10) * ry);
}

/* lgamma of a DD y > 0 (finite, y.x < 2^1014) */
static dd_t lgamma_pos(dd_t y) {
  if (y.x >= 8) return lg_stirling(y);
  if (y.x >= 1.75 && y.x < 2.5) return lg_r2(ddnormalize_d2_d2(ddadd2_d2_d2_d(y, -2.0)));
  if (y.x >= 1.25 && y.x < 1.75) return lg_m(ddnormalize_d2_d2(ddadd2_d2_d2_d(y, -1.5)));
  if (y.x >= 0.5 && y.x < 1.25) {
    dd_t r = y.x < 0.75 ? lg_m(ddnormalize_d2_d2(ddadd2_d2_d2_d(y, -0.5)))
                        : lg_r2(ddnormalize_d2_d2(ddadd2_d2_d2_d(y, -1.0)));
    dd_t l = oracle_logk_dd(y);
    return ddadd2_d2_d2_d2(r, dd(-l.x, -l.y));
  }
  int n = (int)(8.0 - floor(y.x));            /* y + n in [8, 9) */
  dd_t P = y, z = y;
  for (int i = 1; i < n; i++) {
    z = ddadd2_d2_d2_d(z, 1.0);
    P = ddmul_d2_d2_d2(P, z);
  }
  dd_t s = lg_stirling(ddadd2_d2_d2_d(y, (double)n));
  dd_t l = oracle_logk_dd(P);
  return ddadd2_d2_d2_d2(s, dd(-l.x, -l.y));
}

/* sin(pi x) as a DD for finite x with |x| < 2^52 */
static dd_t sinpi_dd(double x) {
  double r = x - 2.0 * rint(0.5 * x);            /* [-1, 1], exact */
  double s = r > 0.5 ? 1.0 - r : (r < -0.5 ? -1.0 - r : r);   /* [-1/2, 1/2], exact */
  dd_t T = ddmul_d2_d_d(s, s);
  double p = poly_d(T.x, SP_P, 11);
  dd_t in = ddadd2_d2_d2_d(dd(SP_H[0], SP_H[1]), T.x * p);
  in = ddadd2_d2_d2_d2(dd(PI_H, PI_L), ddmul_d2_d2_d2(T, in));
  return ddmul_d2_d2_d(in, s);
}

/* log-gamma as a DD and the sign of gamma for finite non-integer-or-positive x */
static dd_t lgamma_dd(double x, int *sign) {
  *sign = 1;
  if (x > 0) return lgamma_pos(dd(x, 0.0));
  /* |x| < 2^-900: sin(pi x) is pi x to far below an ulp, and pi x itself
   * would lose its precision in the subnormal range; it is formed from
   * x 2^200 (exact) and 200 ln 2 is taken off its logarithm */
  int up = fabs(x) < 0x1p-900;
  dd_t sp = up ? ddmul_d2_d2_d(dd(PI_H, PI_L), ldexp(x, 200)) : sinpi_dd(x);
  *sign = sp.x < 0 ? -1 : 1;
  dd_t l = oracle_logk_dd(dd(fabs(sp.x), sp.x < 0 ? -sp.y : sp.y));
  if (up) l = ddadd2_d2_d2_d2(l, dd(-LN2X200_H, -LN2X200_L));
  dd_t r = ddadd2_d2_d2_d2(dd(LOGPI_H, LOGPI_L), dd(-l.x, -l.y));
  dd_t g = lgamma_pos(ddadd2_d2_d_d(1.0, -x));
  return ddadd2_d2_d2_d2(r, dd(-g.x, -g.y));
}

double oracle_lgamma_u10_f64(double x) {
  double a = fabs(x);
  int sign;
  double y;
  if (isnan(x)) return canon_nan();
  if (isinf(x) || x == 0 || (x < 0 && (a >= 0x1p52 || x == rint(x)))) return INFINITY;
  if (x > 0x1p1015) return INFINITY;            /* lgamma overflows from 2.5563e305 */
  dd_t L = lgamma_dd(x, &sign);
  y = L.x + L.y;
  if (!isfinite(y)) y = INFINITY;
  return canon(y);
}

double oracle_tgamma_u10_f64(double x) {
  double a = fabs(x);
  if (isnan(x) || x == -INFINITY || (x < 0 && (a >= 0x1p52 || x == rint(x)))) return canon_nan();
  if (x == 0) return copysign(INFINITY, x);
  if (x > 172) return INFINITY;
  if (x < -190) {
    /* |gamma(x)| < 2^-1100: +-0 with the sign of sin(pi x) */
    dd_t sp = sinpi_dd(x);
    return sp.x < 0 ? -0.0 : 0.0;
  }
  if (x > 0) return canon(oracle_exp_dd(lgamma_pos(dd(x, 0.0))));
  /* x < 0: the reflection in linear form, gamma(x) = pi / (sin(pi x) gamma(1-x))
   * with gamma(1-x) = e^g, g = lgamma(1-x) > -0.13: e^-g = 2^k (1 + s) from the
   * DD exp core, pi (1 + s) / |sin(pi x)| in DD, then 2^k applied once */
  /* |x| < 2^-900: sin(pi x) is pi x to far below an ulp; it is formed from
   * x 2^200 (exact) so that it keeps full precision where pi x would be
   * subnormal, and the quotient gets 2^-200 back with 2^k */
  int up = fabs(x) < 0x1p-900 ? 200 : 0;
  dd_t sp = up ? ddmul_d2_d2_d(dd(PI_H, PI_L), ldexp(x, 200)) : sinpi_dd(x);
  int neg = sp.x < 0;
  dd_t d = dd(fabs(sp.x), neg ? -sp.y : sp.y);
  dd_t g = lgamma_pos(ddadd2_d2_d_d(1.0, -x));
  double k;
  dd_t e = ddadd_d2_d_d2(1.0, oracle_expk_s(dd(-g.x, -g.y), &k));
  dd_t q = dddiv_d2_d2_d2(ddmul_d2_d2_d2(dd(PI_H, PI_L), e), d);
  double y = oracle_scale2(q.x + q.y, (int)k + up);   /* +inf when it overflows */
  return canon(neg ? -y : y);
}

double oracle_lgamma_u35_f64(double x) { return oracle_lgamma_u10_f64(x); }
double oracle_tgamma_u35_f64(double x) { return oracle_tgamma_u10_f64(x); }
