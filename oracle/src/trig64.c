/*
 * FP64 sin, cos, tan and sincos of the oracle, 1-ULP (u10) and 3.5-ULP (u35).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * Structure (Sections 5.1, 5.2, 5.8, Appendix A):
 *   |x| < 15      Cody-Waite level 1: the two-constant split of pi/2 printed
 *                 in the tan listing (fma with the head, DD add of the tail);
 *   |x| < 1e14    Cody-Waite level 2 (constants not printed; this design):
 *                 head by fma (exact), second constant by an exact DD product,
 *                 third constant folded into the tail;
 *   otherwise     the vectorizable Payne-Hanek reduction of Section 5.8, which
 *                 also absorbs non-finite inputs (head set to NaN).
 * Every reduction yields a quarter-turn count q and s = x - q pi/2 as DD.
 * sin and cos use one sine polynomial on [-pi/2, pi/2] (q forced even for sin
 * and odd for cos); tan follows the Appendix A listing; sincos shares one
 * quarter-turn reduction between a sine and a cosine polynomial.
 */
#include "common.h"

#define PIO2_A 0x1.921fb54442d18p0        /* Appendix A listing */
#define PIO2_B 0x1.1a62633145c07p-54      /* Appendix A listing */
#define PIO2_C (-0x1.f1976b7ed8fbcp-110)  /* RN(pi/2 - A - B) */
#define TWOPI_H 0x1.921fb54442d18p2       /* Appendix A listing */
#define TWOPI_L 0x1.1a62633145c07p-52
#define R_1_PI 0x1.45f306dc9c883p-2       /* RN(1/pi) */
#define R_2_PI 0x1.45f306dc9c883p-1       /* RN(2/pi), M_2_PI */

extern const double *oracle_ph_tab(void);
extern const uint8_t *oracle_ph_ibit(void);

/* Section 5.8 / Appendix A: returns 2 pi * rfrac-reduced turns as a DD in
 * [-pi/4, pi/4] and the quarter-turn count mod 4 in *q.
 * The table drops M*I(E)/2 turns; a half turn is put back through q when the
 * mantissa and I(E) are both odd.
 * Each of the four steps of Eq. (ph0) adds M*F_i(E) (the first to zero, so
 * the product itself), takes r = round(4 x.hi) quarter turns off the head
 * (x.hi - r/4, exact, one fma) and renormalizes.  Only q mod 4 is used by
 * the callers, and the paper's per-step increment r - 4 round(x.hi) is r
 * mod 4, so q takes the two low bits of the integer r; 4 x.hi is an exact
 * exponent step. */
dd_t oracle_ph_reduce_dd(double d, int *qo) {
  const double *tab = oracle_ph_tab();
  double df = isfinite(d) ? d : 0.0;
  int ex = ilogb(df), M = ex > 700 ? -130 : -2;
  if (ex < 0) ex = 0;
  if (ex > 1023) ex = 1023;
  double u = ldexp(df, M);
  dd_t x = dd(0, 0);
  int q = 0;
  for (int i = 0; i < 4; i++) {
    dd_t y = ddmul_d2_d_d(u, tab[ex * 4 + i]);
    x = i == 0 ? y : ddadd2_d2_d2_d2(x, y);
    double r = rint(ldexp(x.x, 2));
    q += low2_of_integral(r);
    x.x = fma(r, -0.25, x.x);
    x = ddnormalize_d2_d2(x);
  }
  x = ddmul_d2_d2_d2(x, dd(TWOPI_H, TWOPI_L));
  q += 2 * (int)(dbits(df) & oracle_ph_ibit()[ex] & 1);
  if (!isfinite(d)) x.x = NAN;
  *qo = q & 3;
  return x;
}

/* level-1 Cody-Waite with quarter count qd (Appendix A listing) */
static dd_t cw1(double x, double qd) {
  double u = fma(qd, -PIO2_A, x);
  return ddadd_d2_d_d(u, qd * -PIO2_B);
}
/* level-1 form for cos at |x| < 1 (q = +-1): there x is finer-grained than
 * x - q A, so the fma head is not exact; q A is taken as an exact DD product
 * and added with TwoSum instead */
static dd_t cw1_exact(double x, double qd) {
  dd_t s = ddadd2_d2_d_d2(x, ddmul_d2_d_d(qd, -PIO2_A));
  return ddadd_d2_d2_d(s, qd * -PIO2_B);
}
/* level-2 Cody-Waite for |x| < 1e14: x - qd*A is exact, qd*B is an exact
 * DD product, qd*C goes into the tail */
static dd_t cw2(double x, double qd) {
  double u = fma(qd, -PIO2_A, x);
  dd_t h = ddmul_d2_d_d(qd, -PIO2_B);
  dd_t s = ddadd2_d2_d_d2(u, h);
  s.y = fma(qd, -PIO2_C, s.y);
  return s;
}
/* u35 reductions: same constants, double-only accumulation */
static double cw1_d(double x, double qd) { return fma(qd, -PIO2_B, fma(qd, -PIO2_A, x)); }
static double cw2_d(double x, double qd) {
  return fma(qd, -PIO2_C, fma(qd, -PIO2_B, fma(qd, -PIO2_A, x)));
}
static int q_of(double qd) { return (int)((int64_t)qd & 3); }

/* Section 5.1 uses a half-turn grid: move a Payne-Hanek quarter-turn result
 * with the wrong parity by +-pi/2 so that |s| <= pi/2 (parity 0: sin, 1: cos) */
static dd_t ph_fold(dd_t r, int *q, int parity) {
  if ((*q & 1) != parity) {
    double sg = r.x >= 0 ? -1.0 : 1.0;
    r = ddadd_d2_d2_d2(dd(sg * PIO2_A, sg * PIO2_B), r);
    *q -= (int)sg;
  }
  return r;
}

/* ---------------- sin / cos, u10 ---------------- */
static const double SIN_C1H = -0x1.5555555555555p-3, SIN_C1L = 0x1.07fb00106bcfdp-57;
static const double SIN_U10[7] = {
  0x1.111111111109fp-7, -0x1.a01a01a0129ddp-13, 0x1.71de3a51b383dp-19,
  -0x1.ae64546a1a9ebp-26, 0x1.6123b2c07aaa7p-33, -0x1.ae3cc8078333ap-41,
  0x1.877f977ffe028p-49 };

/* sin s = s + s t (c1 + t P(t)), t = s^2; c1 and the two products in DD */
static double sin_poly_u10(dd_t s) {
  dd_t t = ddsqu_d2_d2(s);
  double p = poly_d(t.x, SIN_U10, 7);
  dd_t w = ddadd_d2_d2_d(dd(SIN_C1H, SIN_C1L), t.x * p);
  w = ddmul_d2_d2_d2(t, w);
  w = ddmul_d2_d2_d2(s, w);
  dd_t r = ddadd_d2_d2_d2(s, w);
  return r.x + r.y;
}

/* half-turn reduction for sin (parity 0) or cos (parity 1) */
static dd_t reduce_half(double x, int parity, int *q) {
  double ax = fabs(x);
  if (ax < 1e14) {
    double qd = parity ? 2.0 * rint(fma(x, R_1_PI, -0.5)) + 1.0 : 2.0 * rint(x * R_1_PI);
    *q = q_of(qd);
    if (parity && ax < 1) return cw1_exact(x, qd);
    return ax < 15 ? cw1(x, qd) : cw2(x, qd);
  }
  dd_t r = oracle_ph_reduce_dd(x, q);
  return ph_fold(r, q, parity);
}

double oracle_sin_u10_f64(double x) {
  int q;
  dd_t s = reduce_half(x, 0, &q);
  double y = sin_poly_u10(s);
  if (q & 2) y = -y;
  if (x == 0) y = x;
  return canon(y);
}

double oracle_cos_u10_f64(double x) {
  int q;
  dd_t s = reduce_half(x, 1, &q);
  double y = sin_poly_u10(s);
  if (!(q & 2)) y = -y;
  return canon(y);
}

/* ---------------- sin / cos, u35 ---------------- */
static const double SIN_U35[8] = {
  -0x1.5555555555555p-3, 0x1.11111111110bdp-7, -0x1.a01a01a013e17p-13,
  0x1.71de3a5220856p-19, -0x1.ae645492b5795p-26, 0x1.6123bb419f3c8p-33,
  -0x1.ae3ea885fb135p-41, 0x1.87ab1397c30b7p-49 };

static double reduce_half_d(double x, int parity, int *q) {
  double ax = fabs(x);
  if (ax < 1e14) {
    double qd = parity ? 2.0 * rint(fma(x, R_1_PI, -0.5)) + 1.0 : 2.0 * rint(x * R_1_PI);
    *q = q_of(qd);
    return ax < 15 ? cw1_d(x, qd) : cw2_d(x, qd);
  }
  dd_t r = oracle_ph_reduce_dd(x, q);
  r = ph_fold(r, q, parity);
  return r.x + r.y;
}

static double sin_poly_u35(double s) {
  double t = s * s;
  return fma(s * t, poly_d(t, SIN_U35, 8), s);
}

double oracle_sin_u35_f64(double x) {
  int q;
  double s = reduce_half_d(x, 0, &q);
  double y = sin_poly_u35(s);
  if (q & 2) y = -y;
  if (x == 0) y = x;
  return canon(y);
}

double oracle_cos_u35_f64(double x) {
  int q;
  double s = reduce_half_d(x, 1, &q);
  double y = sin_poly_u35(s);
  if (!(q & 2)) y = -y;
  return canon(y);
}

/* ---------------- quarter-turn reduction (tan, sincos) ---------------- */
static dd_t reduce_quarter(double x, int *q) {
  double ax = fabs(x);
  if (ax < 1e14) {
    double qd = rint(x * R_2_PI);
    *q = q_of(qd);
    return ax < 15 ? cw1(x, qd) : cw2(x, qd);
  }
  return oracle_ph_reduce_dd(x, q);
}
static double reduce_quarter_d(double x, int *q) {
  double ax = fabs(x);
  if (ax < 1e14) {
    double qd = rint(x * R_2_PI);
    *q = q_of(qd);
    return ax < 15 ? cw1_d(x, qd) : cw2_d(x, qd);
  }
  dd_t r = oracle_ph_reduce_dd(x, q);
  return r.x + r.y;
}

/* ---------------- tan (Section 5.2, Appendix A listing) ---------------- */
/* the listing's ESTRIN coefficients, constant term first */
static const double TAN_C[8] = {
  +0.1333333333330500581e+0, +0.5396825399517272970e-1, +0.2186948728185535498e-1,
  +0.8863268409563113126e-2, +0.3591611540792499519e-2, +0.1460781502402784494e-2,
  +0.5619219738114323735e-3, +0.3245098826639276316e-3 };
static const double TAN_C3 = +0.3333333333333343695e+0;

double oracle_tan_u10_f64(double d) {
  int q;
  dd_t x = reduce_quarter(d, &q), y;
  y = ddscale_d2_d2_d(x, 0.5);                 /* double-angle reduction */
  x = ddsqu_d2_d2(y);
  double u = poly_d(x.x, TAN_C, 8);
  u = fma(u, x.x, TAN_C3);
  x = ddadd_d2_d2_d2(y, ddmul_d2_d2_d(ddmul_d2_d2_d2(x, y), u));
  y = ddadd_d2_d_d2(-1, ddsqu_d2_d2(x));       /* reconstruction */
  x = ddscale_d2_d2_d(x, -2);
  if (q & 1) { dd_t t = x; x = y; y = dd(-t.x, -t.y); }
  x = dddiv_d2_d2_d2(x, y);
  double r = x.x + x.y;
  if (d == 0) r = d;
  return canon(r);
}

/* a / b within about a unit of the correctly rounded quotient (reading
 * R35): the reciprocal of b's significand from its binary32 reciprocal
 * (significand truncated to 24 bits, exact widening) and two Newton steps
 * with fma, scaled by 2^-ilogb|b|, the quotient a r and one fma correction
 * q + (a - q b) r; b outside [2^-1000, 2^1000] (zero, subnormal, huge, not
 * finite) takes the IEEE division */
static double div_u35(double a, double b) {
  double ab = fabs(b);
  if (!(ab >= 0x1p-1000 && ab <= 0x1p1000)) return a / b;
  uint64_t bb = dbits(ab), man = bb & 0x000FFFFFFFFFFFFFULL;
  int e = (int)(bb >> 52) - 1023;
  uint64_t mb = 0x3FF0000000000000ULL | man;
  uint32_t fb = 0x3F800000U | (uint32_t)(man >> 29);
  double m;
  float mf;
  memcpy(&m, &mb, 8);
  memcpy(&mf, &fb, 4);
  float rf = 1.0f / mf;
  uint32_t rb = fbits(rf);
  uint64_t yb = ((uint64_t)((rb >> 23) + 896) << 52) | ((uint64_t)(rb & 0x7FFFFF) << 29);
  double y;
  memcpy(&y, &yb, 8);
  double t = fma(-m, y, 1.0);
  y = fma(y, t, y);
  t = fma(-m, y, 1.0);
  y = fma(y, t, y);                                         /* 1/m to about an ulp */
  uint64_t rbits = dbits(y) - ((uint64_t)(int64_t)e << 52);
  double r;
  memcpy(&r, &rbits, 8);
  if (b < 0) r = -r;
  double q = a * r;
  return fma(fma(-q, b, a), r, q);
}

/* u35: the same polynomial in double, one division for the reconstruction */
double oracle_tan_u35_f64(double d) {
  int q;
  double s = reduce_quarter_d(d, &q);
  double y = s * 0.5, t = y * y;
  double u = fma(poly_d(t, TAN_C, 8), t, TAN_C3);
  double tt = fma(y * t, u, y);
  double num = tt + tt, den = fma(-tt, tt, 1.0);
  double r = (q & 1) ? div_u35(-den, num) : div_u35(num, den);
  if (d == 0) r = d;
  return canon(r);
}

/* ---------------- sincos ---------------- */
static const double SC_S1H = -0x1.5555555555543p-3, SC_S1L = 0x1.cc5eebaea7e3cp-57;
static const double SC_S_U10[5] = {
  0x1.111111110eea5p-7, -0x1.a01a019ad6669p-13, 0x1.71de3466b0f92p-19,
  -0x1.ae5d912c0cb21p-26, 0x1.5d558cd2a4be1p-33 };
static const double SC_C[6] = {
  0x1.5555555555546p-5, -0x1.6c16c16c14555p-10, 0x1.a01a019b8491fp-16,
  -0x1.27e4f73296656p-22, 0x1.1ee95b26826a1p-29, -0x1.8f6489336e5adp-37 };
static const double SC_S_U35[6] = {
  -0x1.5555555555543p-3, 0x1.111111110ef1dp-7, -0x1.a01a019ae1837p-13,
  0x1.71de346e3d979p-19, -0x1.ae5d95f8b7e3ep-26, 0x1.5d56b550f4cf7p-33 };

static void sc_quadrant(int q, double *sn, double *cs) {
  if (q & 1) { double t = *sn; *sn = *cs; *cs = -t; }
  if (q & 2) { *sn = -*sn; *cs = -*cs; }
}

void oracle_sincos_u10_f64(double d, double *ps, double *pc) {
  int q;
  dd_t s = reduce_quarter(d, &q);
  dd_t t = ddsqu_d2_d2(s);
  double p = poly_d(t.x, SC_S_U10, 5);
  dd_t w = ddadd_d2_d2_d(dd(SC_S1H, SC_S1L), t.x * p);
  w = ddmul_d2_d2_d2(t, w);
  w = ddmul_d2_d2_d2(s, w);
  dd_t rs = ddadd_d2_d2_d2(s, w);
  double sn = rs.x + rs.y;
  double pcv = poly_d(t.x, SC_C, 6);
  dd_t h = ddadd_d2_d_d2(1.0, ddscale_d2_d2_d(t, -0.5));
  h = ddadd_d2_d2_d(h, (t.x * t.x) * pcv);
  double cs = h.x + h.y;
  sc_quadrant(q, &sn, &cs);
  if (d == 0) sn = d;
  *ps = canon(sn);
  *pc = canon(cs);
}

void oracle_sincos_u35_f64(double d, double *ps, double *pc) {
  int q;
  double s = reduce_quarter_d(d, &q);
  double t = s * s;
  double sn = fma(s * t, poly_d(t, SC_S_U35, 6), s);
  double cs = fma(t, fma(t, poly_d(t, SC_C, 6), -0.5), 1.0);
  sc_quadrant(q, &sn, &cs);
  if (d == 0) sn = d;
  *ps = canon(sn);
  *pc = canon(cs);
}
