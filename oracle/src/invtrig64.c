/*
 * FP64 asin, acos, atan and atan2 of the oracle, u10 and u35.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * asin/acos (Section 5.3): |x| <= 0.5 directly; otherwise through
 *   asin x = pi/2 - 2 asin(sqrt((1-x)/2)) and acos x = 2 asin(sqrt((1-x)/2))
 *   (pi - ... for x < -0.5); one arcsine polynomial on [0, 0.5].
 * atan (Section 5.4): a' = 1/a if |a| >= 1; one polynomial on [0, 1];
 *   atan a = pi/2 - atan a' in that case.
 * atan2 (the paper names it only among the C99 functions): the quotient of
 *   the smaller by the larger magnitude in DD, the atan core, then pi/2 - r
 *   and pi - r reconstructions; C99 Annex F special pairs are selected last.
 */
#include "common.h"
#include "coeffs64.h"

#define PIO2H 0x1.921fb54442d18p0
#define PIO2L 0x1.1a62633145c07p-54
#define PIH 0x1.921fb54442d18p1
#define PIL 0x1.1a62633145c07p-53
#define PI4 0x1.921fb54442d18p-1
#define PI34 0x1.2d97c7f3321d2p1

static const double ASIN_U10[13] = { ASIN_U10_COEFFS };
static const double AT_C1H = ATAN_U10_C1H, AT_C1L = ATAN_U10_C1L;
static const double ATAN_U10[20] = { ATAN_U10_COEFFS };
static const double ATAN_U35[19] = { ATAN_U35_COEFFS };

/* sqrt of a non-negative double as DD; the tail is 0 for a zero argument */
static dd_t sqrt_dd(double t) {
  double h = sqrt(t);
  double r = fma(-h, h, t);
  double lo = r * (1.0 / (h + h));
  return dd(h, h > 0 ? lo : 0.0);
}

/* asin(u) as DD for u = |x| (|x| <= 0.5) or sqrt((1-|x|)/2) */
static dd_t asin_core_u10(double ax) {
  dd_t u;
  double t;
  if (ax <= 0.5) { u = dd(ax, 0); t = ax * ax; }
  else { t = (1.0 - ax) * 0.5; u = sqrt_dd(t); }
  double corr = (u.x * t) * poly_d(t, ASIN_U10, 13);
  return ddadd_d2_d2_d(u, corr);
}

double oracle_asin_u10_f64(double x) {
  double ax = fabs(x);
  dd_t r = asin_core_u10(ax);
  if (ax > 0.5) r = ddadd_d2_d2_d2(dd(PIO2H, PIO2L), ddscale_d2_d2_d(r, -2.0));
  double y = copysign(r.x + r.y, x);
  if (ax > 1) y = NAN;
  return canon(y);
}

double oracle_acos_u10_f64(double x) {
  double ax = fabs(x);
  dd_t r = asin_core_u10(ax), s;
  if (ax <= 0.5) s = ddadd_d2_d2_d2(dd(PIO2H, PIO2L), x < 0 ? r : dd(-r.x, -r.y));
  else if (x > 0) s = ddscale_d2_d2_d(r, 2.0);
  else s = ddadd_d2_d2_d2(dd(PIH, PIL), ddscale_d2_d2_d(r, -2.0));
  double y = s.x + s.y;
  if (ax > 1) y = NAN;
  return canon(y);
}

static double asin_core_u35(double ax) {
  double u, t;
  if (ax <= 0.5) { u = ax; t = ax * ax; }
  else { t = (1.0 - ax) * 0.5; u = sqrt(t); }
  return fma(u * t, poly_d(t, ASIN_U10, 13), u);
}

double oracle_asin_u35_f64(double x) {
  double ax = fabs(x);
  double r = asin_core_u35(ax);
  if (ax > 0.5) r = fma(-2.0, r, PIO2H) + PIO2L;
  double y = copysign(r, x);
  if (ax > 1) y = NAN;
  return canon(y);
}

double oracle_acos_u35_f64(double x) {
  double ax = fabs(x);
  double r = asin_core_u35(ax), y;
  if (ax <= 0.5) y = (PIO2H - copysign(r, x)) + PIO2L;
  else if (x > 0) y = 2.0 * r;
  else y = fma(-2.0, r, PIH) + PIL;
  if (ax > 1) y = NAN;
  return canon(y);
}

/* atan(s) as DD for s in [0, 1] given as DD: s + s t (c1 + t P(t)) */
static dd_t atan_core_u10(dd_t s) {
  dd_t t = ddsqu_d2_d2(s);
  double p = poly_d(t.x, ATAN_U10, 20);
  dd_t w = ddadd_d2_d2_d(dd(AT_C1H, AT_C1L), t.x * p);
  w = ddmul_d2_d2_d2(t, w);
  w = ddmul_d2_d2_d2(s, w);
  return ddadd_d2_d2_d2(s, w);
}

double oracle_atan_u10_f64(double x) {
  double ax = fabs(x);
  dd_t s = ax >= 1 ? ddrec_d2_d(ax) : dd(ax, 0);
  if (isinf(x)) s = dd(0, 0);
  dd_t r = atan_core_u10(s);
  if (ax >= 1) r = ddadd_d2_d2_d2(dd(PIO2H, PIO2L), dd(-r.x, -r.y));
  return canon(copysign(r.x + r.y, x));
}

static double atan_core_u35(double s) {
  double t = s * s;
  return fma(s * t, poly_d(t, ATAN_U35, 19), s);
}

double oracle_atan_u35_f64(double x) {
  double ax = fabs(x);
  double s = ax >= 1 ? 1.0 / ax : ax;
  double r = atan_core_u35(s);
  if (ax >= 1) r = PIO2H - r;
  return canon(copysign(r, x));
}

/* Annex F special pairs of atan2(a, b); returns 1 and sets *y if (a, b) is one */
static int atan2_special(double a, double b, double *y) {
  if (isnan(a) || isnan(b)) { *y = NAN; return 1; }
  if (isinf(b)) {
    if (isinf(a)) *y = copysign(b > 0 ? PI4 : PI34, a);
    else *y = copysign(b > 0 ? 0.0 : PIH, a);
    return 1;
  }
  if (isinf(a)) { *y = copysign(PIO2H, a); return 1; }
  if (a == 0 && b == 0) { *y = copysign(signbit(b) ? PIH : 0.0, a); return 1; }
  return 0;
}

double oracle_atan2_u10_f64(double a, double b) {
  double aa = fabs(a), ab = fabs(b);
  int swap = aa > ab;
  double num = swap ? ab : aa, den = swap ? aa : ab;
  if (!(den > 0 && den <= 0x1.fffffffffffffp1023) || !(num <= den)) { num = 0.0; den = 1.0; }
  if (den < 0x1p-1000) { num *= 0x1p600; den *= 0x1p600; }      /* keep 1/den finite */
  if (den > 0x1p1000) { num *= 0x1p-600; den *= 0x1p-600; }     /* keep 1/den normal */
  dd_t s = dddiv_d2_d2_d2(dd(num, 0), dd(den, 0));
  dd_t r = atan_core_u10(s);
  if (swap) r = ddadd_d2_d2_d2(dd(PIO2H, PIO2L), dd(-r.x, -r.y));
  if (b < 0) r = ddadd_d2_d2_d2(dd(PIH, PIL), dd(-r.x, -r.y));
  double y = copysign(r.x + r.y, a);
  atan2_special(a, b, &y);
  return canon(y);
}

double oracle_atan2_u35_f64(double a, double b) {
  double aa = fabs(a), ab = fabs(b);
  int swap = aa > ab;
  double num = swap ? ab : aa, den = swap ? aa : ab;
  if (!(den > 0 && den <= 0x1.fffffffffffffp1023) || !(num <= den)) { num = 0.0; den = 1.0; }
  if (den < 0x1p-1000) { num *= 0x1p600; den *= 0x1p600; }      /* keep 1/den finite */
  if (den > 0x1p1000) { num *= 0x1p-600; den *= 0x1p-600; }     /* keep 1/den normal */
  double r = atan_core_u35(num * (1.0 / den));
  if (swap) r = PIO2H - r;
  if (b < 0) r = PIH - r;
  double y = copysign(r, a);
  atan2_special(a, b, &y);
  return canon(y);
}
