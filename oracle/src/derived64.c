/*
 * FP64 functions of the oracle that the paper does not describe step by
 * step (it names them as part of the library but gives algorithms only for
 * the core functions): exp2, exp10, expm1, log2, log10, log1p, cbrt, sinh,
 * cosh, tanh, asinh, acosh, atanh, each in a 1-ULP (u10) and a 3.5-ULP (u35)
 * form.  They are built from the exp and log cores of Sections 5.5-5.6 with
 * the DD arithmetic of Section 3; every step is plain IEEE arithmetic with
 * explicit fma(), so the CUDA kernels can repeat it bit for bit.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * Parity is pinned by the __float128 ULP bounds, C99 Annex F special values
 * and identities (exp2(k) = 2^k, cbrt(8) = 2, log2(2^k) = k, ...); the op
 * sequences themselves are this library's design.
 *
 * exp2   k = rint(x), r = x - k exact, r ln2 as a DD, then the exp tail.
 * exp10  k = rint(x log2 10), r = x - k log10(2) with a two-part constant
 *        (head exact), r ln10 as a DD, then the exp tail.
 * expm1  e^x - 1 = 2^k s + (2^k - 1) with s = e^r - 1 as a DD: no
 *        cancellation at k = 0 and exact 2^k - 1 elsewhere.
 * log2, log10, log1p   the log core on a DD argument (1 + x exactly for
 *        log1p), the result multiplied by DD constants (u10) or the core
 *        rounded to double and multiplied in double (u35).
 * cbrt   a = m 2^(3q + i) with a in [1, 8); a^(-1/3) from a polynomial and
 *        one Newton step without division; y = a z^2 and one Newton step on
 *        y whose residual y^3 - a is exact in DD (u10) or rounded (u35).
 * sinh, cosh, tanh   from e^|x| - 1 in DD (sinh = (e + e/(e+1))/2,
 *        cosh = (E + 1/E)/2, tanh = e2/(e2 + 2) with e2 = e^(2|x|) - 1);
 *        for large |x| e^|x|/2 directly.
 * asinh, acosh, atanh   log of the DD argument |x| + sqrt(x^2 + 1),
 *        x + sqrt((x-1)(x+1)), (1+|x|)/(1-|x|): the DD logarithm (u10), or
 *        the logarithm in double with its z corrected once (u35).
 */
#include "common.h"
#include "coeffs64.h"
#include "explog64.h"

#define R_LN2 0x1.71547652b82fep+0
#define L2A 0x1.62e42fefa39efp-1       /* RN(ln2) */
#define L2B 0x1.abc9e3b39803fp-56      /* RN(ln2 - L2A) */
#define L2H 0x1.62e42fefa3800p-1       /* ln2 to 42 bits: e L2H exact for |e| < 2^11 */
#define L2L 0x1.ef35793c76730p-45
#define RL2H 0x1.71547652b82fep+0      /* 1/ln2 as a DD */
#define RL2L 0x1.777d0ffda0d24p-56
#define RL10H 0x1.bcb7b1526e50ep-2     /* 1/ln10 as a DD */
#define RL10L 0x1.95355baaafad3p-57
#define LN10H 0x1.26bb1bbb55516p+1     /* ln10 as a DD */
#define LN10L -0x1.f48ad494ea3e9p-53
#define LOG2_10 0x1.a934f0979a371p+1   /* RN(log2 10) */
#define L10A 0x1.34413509f79ffp-2      /* RN(log10 2) */
#define L10B -0x1.9dc1da994fd21p-59    /* RN(log10 2 - L10A) */
#define LG2H 0x1.34413509f7800p-2      /* log10 2 to 42 bits */
#define LG2L 0x1.fef311f12b358p-46
#define THIRD 0x1.5555555555555p-2
#define TWO_M28 0x1p-28

static const double EXPM1_U35[10] = { EXPM1_U35_COEFFS };
static const double CBRT_P[8] = { CBRT_COEFFS };
static const double CBRT_C[3] = { 1.0, 0x1.965fea53d6e3dp-1, 0x1.428a2f98d728bp-1 };  /* RN(2^(-i/3)) */

/* e^t - 1 for |t| <= ln2/2 with the polynomial fitted relative to e^t - 1
 * (12 terms), rounded once by the last fma */
static double em1_r_u35(double t) { return fma(t * t, poly_d(t, EXPM1_U35, 10), t); }

/* ---------------- exp2, exp10 ---------------- */
double oracle_exp2_u10_f64(double x) {
  double xc = fabs(x) <= 1100 ? x : 0.0;
  double k = rint(xc);
  double r = xc - k;
  dd_t t = ddmul_d2_d2_d(dd(L2A, L2B), r);
  double y = oracle_exp_tail_u10(t.x, t.y, k);
  if (!(fabs(x) <= 1100)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}

double oracle_exp2_u35_f64(double x) {
  double xc = fabs(x) <= 1100 ? x : 0.0;
  double k = rint(xc);
  double t = (xc - k) * L2A;
  double y = oracle_scale2(1.0 + em1_r_u35(t), (int)k);
  if (!(fabs(x) <= 1100)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}

double oracle_exp10_u10_f64(double x) {
  double xc = fabs(x) <= 350 ? x : 0.0;
  double k = rint(xc * LOG2_10);
  double h = fma(k, -L10A, xc);
  double r = fma(k, -L10B, h);
  double rl = fma(k, -L10B, h - r);
  dd_t t = ddmul_d2_d2_d2(dd(r, rl), dd(LN10H, LN10L));
  double y = oracle_exp_tail_u10(t.x, t.y, k);
  if (!(fabs(x) <= 350)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}

double oracle_exp10_u35_f64(double x) {
  double xc = fabs(x) <= 350 ? x : 0.0;
  double k = rint(xc * LOG2_10);
  double r = fma(k, -L10B, fma(k, -L10A, xc));
  double y = oracle_scale2(1.0 + em1_r_u35(r * LN10H), (int)k);
  if (!(fabs(x) <= 350)) y = x > 0 ? INFINITY : (x < 0 ? 0.0 : NAN);
  return canon(y);
}

/* ---------------- expm1 ---------------- */
/* e^a - 1 as a DD for -40 < a <= 40: 2^k s + (2^k - 1), the second term an
 * exact DD */
static dd_t em1_dd(double a) {
  double k;
  dd_t s = oracle_expk_s(dd(a, 0.0), &k);
  double p = ldexp(1.0, (int)k);
  return ddadd2_d2_d2_d2(ddadd2_d2_d_d(p, -1.0), ddscale_d2_d2_d(s, p));
}

double oracle_expm1_u10_f64(double x) {
  double xc = (x > -40 && x < 710) ? x : 0.0;
  double k;
  dd_t s = oracle_expk_s(dd(xc, 0.0), &k);
  double y;
  if (k > 1000) {
    dd_t e = ddadd_d2_d_d2(1.0, s);
    y = oracle_scale2(e.x + e.y, (int)k);
  } else {
    double p = ldexp(1.0, (int)k);
    dd_t r = ddadd2_d2_d2_d2(ddadd2_d2_d_d(p, -1.0), ddscale_d2_d2_d(s, p));
    y = r.x + r.y;
  }
  if (x == 0) y = x;
  if (!(x > -40 && x < 710)) y = x >= 710 ? INFINITY : (x <= -40 ? -1.0 : NAN);
  return canon(y);
}

/* u35: e^r - 1 in double with a polynomial fitted relative to e^r - 1
 * (12 terms), then 2^k v + (2^k - 1) with one rounding */
static double em1_u35(double xc, double *kp) {
  double k = rint(xc * R_LN2);
  double r = fma(k, -L2B, fma(k, -L2A, xc));
  *kp = k;
  return em1_r_u35(r);
}

double oracle_expm1_u35_f64(double x) {
  double xc = (x > -40 && x < 710) ? x : 0.0;
  double k;
  double v = em1_u35(xc, &k);
  double y;
  if (k > 1000) {
    y = oracle_scale2(1.0 + v, (int)k);
  } else {
    double p = ldexp(1.0, (int)k);
    y = fma(p, v, p - 1.0);
  }
  if (x == 0) y = x;
  if (!(x > -40 && x < 710)) y = x >= 710 ? INFINITY : (x <= -40 ? -1.0 : NAN);
  return canon(y);
}

/* ---------------- log2, log10, log1p ---------------- */
static double log_special(double x, double y) {
  if (x == 0) return -INFINITY;
  if (x < 0 || isnan(x)) return NAN;
  if (isinf(x)) return INFINITY;
  return y;
}

double oracle_log2_u10_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  dd_t lm = oracle_logm_u10(dd(a, 0.0), &e);
  dd_t p = ddmul_d2_d2_d2(lm, dd(RL2H, RL2L));
  dd_t r = ddadd2_d2_d_d2((double)e, p);
  return canon(log_special(x, r.x + r.y));
}

double oracle_log2_u35_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  dd_t lm = oracle_logm_u10(dd(a, 0.0), &e);
  return canon(log_special(x, fma(lm.x + lm.y, RL2H, (double)e)));
}

double oracle_log10_u10_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  dd_t lm = oracle_logm_u10(dd(a, 0.0), &e);
  dd_t p = ddmul_d2_d2_d2(lm, dd(RL10H, RL10L));
  double ed = (double)e;
  dd_t r = ddadd2_d2_d2_d2(dd(ed * LG2H, ed * LG2L), p);
  return canon(log_special(x, r.x + r.y));
}

double oracle_log10_u35_f64(double x) {
  double a = (x > 0 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  dd_t lm = oracle_logm_u10(dd(a, 0.0), &e);
  return canon(log_special(x, fma((double)e, L10A, (lm.x + lm.y) * RL10H)));
}

/* log a as a DD for a DD a > 0 */
static dd_t log_dd(dd_t a) {
  int e;
  dd_t lm = oracle_logm_u10(a, &e);
  double ed = (double)e;
  return ddadd2_d2_d2_d2(dd(ed * L2H, ed * L2L), lm);
}

static double log1p_special(double x, double y) {
  if (x == -1) return -INFINITY;
  if (x < -1 || isnan(x)) return NAN;
  if (isinf(x)) return INFINITY;
  if (x == 0) return x;
  return y;
}

double oracle_log1p_u10_f64(double x) {
  double xc = (x > -1 && x <= 0x1.fffffffffffffp1023) ? x : 0.0;
  dd_t r = log_dd(ddadd2_d2_d_d(1.0, xc));
  return canon(log1p_special(x, r.x + r.y));
}

double oracle_log1p_u35_f64(double x) {
  double xc = (x > -1 && x <= 0x1.fffffffffffffp1023) ? x : 0.0;
  int e;
  double lm = oracle_logm_u35(ddadd2_d2_d_d(1.0, xc), &e);
  return canon(log1p_special(x, fma((double)e, L2A, lm)));
}

/* ---------------- cbrt ---------------- */
static double cbrt_core(double x, int u10) {
  double a0 = fabs(x);
  int fin = isfinite(x) && x != 0;
  if (!fin) a0 = 1.0;
  int off = 0;
  if (a0 < 0x1p-1022) { a0 *= 0x1p54; off = 18; }
  int e = ilogb(a0);
  int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  int i = e - 3 * q;
  double m = ldexp(a0, -e);                     /* [1, 2), exact */
  double a = m * ldexp(1.0, i);                 /* [1, 8), exact */
  double z = poly_d(m - 1.5, CBRT_P, 8) * CBRT_C[i];
  double z3 = (z * z) * z;
  z = fma(z * fma(-a, z3, 1.0), THIRD, z);      /* Newton step for a^(-1/3) */
  double zz = z * z;
  double y = a * zz;
  double d;
  if (u10) {
    dd_t y3 = ddmul_d2_d2_d(ddmul_d2_d_d(y, y), y);
    d = (y3.x - a) + y3.y;                      /* y^3 - a, head difference exact */
  } else {
    d = fma(y * y, y, -a);
  }
  y = fma(-d, zz * THIRD, y);                   /* Newton step for a^(1/3) */
  y = y * ldexp(1.0, q - off);
  if (!fin) y = x + x;                          /* +-0, +-inf, NaN */
  return canon(copysign(y, x));
}

double oracle_cbrt_u10_f64(double x) { return cbrt_core(x, 1); }
double oracle_cbrt_u35_f64(double x) { return cbrt_core(x, 0); }

/* ---------------- sinh, cosh, tanh ---------------- */
double oracle_sinh_u10_f64(double x) {
  double a = fabs(x);
  double ac = a <= 711 ? a : 0.0;
  double y;
  if (ac > 22) {
    double k;
    dd_t s = oracle_expk_s(dd(ac, 0.0), &k);
    dd_t e = ddadd_d2_d_d2(1.0, s);
    y = oracle_scale2(e.x + e.y, (int)k - 1);
  } else {
    dd_t em = em1_dd(ac);
    dd_t f = dddiv_d2_d2_d2(em, ddadd2_d2_d_d2(1.0, em));
    dd_t h = ddadd2_d2_d2_d2(em, f);
    y = 0.5 * (h.x + h.y);
  }
  if (a < TWO_M28) y = a;
  if (!(a <= 711)) y = isnan(x) ? NAN : INFINITY;
  return canon(copysign(y, x));
}

double oracle_cosh_u10_f64(double x) {
  double a = fabs(x);
  double ac = a <= 711 ? a : 0.0;
  double k;
  dd_t s = oracle_expk_s(dd(ac, 0.0), &k);
  dd_t e = ddadd_d2_d_d2(1.0, s);
  double y;
  if (ac > 22) {
    y = oracle_scale2(e.x + e.y, (int)k - 1);
  } else {
    dd_t E = ddscale_d2_d2_d(e, ldexp(1.0, (int)k));
    dd_t h = ddadd_d2_d2_d2(E, ddrec_d2_d2(E));
    y = 0.5 * (h.x + h.y);
  }
  if (!(a <= 711)) y = isnan(x) ? NAN : INFINITY;
  return canon(y);
}

double oracle_tanh_u10_f64(double x) {
  double a = fabs(x);
  double ac = a <= 20 ? a : 0.0;
  dd_t em = em1_dd(ac + ac);
  dd_t t = dddiv_d2_d2_d2(em, ddadd2_d2_d_d2(2.0, em));
  double y = t.x + t.y;
  if (a < TWO_M28) y = a;
  if (!(a <= 20)) y = isnan(x) ? NAN : 1.0;
  return canon(copysign(y, x));
}

double oracle_sinh_u35_f64(double x) {
  double a = fabs(x);
  double ac = a <= 711 ? a : 0.0;
  double k;
  double v = em1_u35(ac, &k);
  double y;
  if (ac > 22) {
    y = oracle_scale2(1.0 + v, (int)k - 1);
  } else {
    double p = ldexp(1.0, (int)k);
    double em = fma(p, v, p - 1.0);
    y = 0.5 * (em + em * (1.0 / (em + 1.0)));
  }
  if (a < TWO_M28) y = a;
  if (!(a <= 711)) y = isnan(x) ? NAN : INFINITY;
  return canon(copysign(y, x));
}

double oracle_cosh_u35_f64(double x) {
  double a = fabs(x);
  double ac = a <= 711 ? a : 0.0;
  double k;
  double v = em1_u35(ac, &k);
  double y;
  if (ac > 22) {
    y = oracle_scale2(1.0 + v, (int)k - 1);
  } else {
    double E = (1.0 + v) * ldexp(1.0, (int)k);
    y = 0.5 * (E + 1.0 / E);
  }
  if (!(a <= 711)) y = isnan(x) ? NAN : INFINITY;
  return canon(y);
}

double oracle_tanh_u35_f64(double x) {
  double a = fabs(x);
  double ac = a <= 20 ? a : 0.0;
  double k;
  double v = em1_u35(ac + ac, &k);
  double p = ldexp(1.0, (int)k);
  double em = fma(p, v, p - 1.0);
  double y = em * (1.0 / (em + 2.0));
  if (a < TWO_M28) y = a;
  if (!(a <= 20)) y = isnan(x) ? NAN : 1.0;
  return canon(copysign(y, x));
}

/* ---------------- asinh, acosh, atanh ---------------- */
double oracle_asinh_u10_f64(double x) {
  double a = fabs(x);
  double ac = a <= 0x1.fffffffffffffp1023 ? a : 1.0;
  dd_t r;
  if (ac > 0x1p500) {
    r = ddadd2_d2_d2_d2(log_dd(dd(ac, 0.0)), dd(L2A, L2B));
  } else {
    dd_t w = ddsqrt_d2_d2(ddadd2_d2_d2_d(ddmul_d2_d_d(ac, ac), 1.0));
    r = log_dd(ddadd2_d2_d2_d(w, ac));
  }
  double y = r.x + r.y;
  if (a < TWO_M28) y = a;
  if (!(a <= 0x1.fffffffffffffp1023)) y = isnan(x) ? NAN : INFINITY;
  return canon(copysign(y, x));
}

double oracle_acosh_u10_f64(double x) {
  double xc = (x >= 1 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  dd_t r;
  if (xc > 0x1p500) {
    r = ddadd2_d2_d2_d2(log_dd(dd(xc, 0.0)), dd(L2A, L2B));
  } else {
    dd_t d = ddmul_d2_d2_d2(ddadd2_d2_d_d(xc, -1.0), ddadd2_d2_d_d(xc, 1.0));
    r = log_dd(ddadd2_d2_d2_d(ddsqrt_d2_d2(d), xc));
  }
  double y = r.x + r.y;
  if (xc == 1) y = 0.0;                         /* the DD square root of 0 is not defined */
  if (!(x >= 1 && x <= 0x1.fffffffffffffp1023)) y = x == INFINITY ? INFINITY : NAN;
  return canon(y);
}

double oracle_atanh_u10_f64(double x) {
  double a = fabs(x);
  double ac = a < 1 ? a : 0.5;
  dd_t q = dddiv_d2_d2_d2(ddadd2_d2_d_d(1.0, ac), ddadd2_d2_d_d(1.0, -ac));
  dd_t r = log_dd(q);
  double y = 0.5 * (r.x + r.y);
  if (a < TWO_M28) y = a;
  if (!(a < 1)) y = a == 1 ? INFINITY : NAN;
  return canon(copysign(y, x));
}

/* 3.5-ULP forms: the same DD arguments as the 1-ULP forms (they carry the
 * cancellation in x^2 + 1 - 1, x^2 - 1 and 1 - |x|), whose logarithm is
 * taken in double with z corrected once (oracle_logm_u20) and e ln 2 added by
 * one fma, instead of the DD logarithm (the plain 3.5-ULP core, z rounded
 * three times, reached 4.0 ULP on asinh near 0.24).
 * Above 2^500, log(2x) = (e + 1) ln 2 + log m. */
double oracle_asinh_u35_f64(double x) {
  double a = fabs(x);
  double ac = a <= 0x1.fffffffffffffp1023 ? a : 1.0;
  int e;
  double lm;
  if (ac > 0x1p500) {
    lm = oracle_logm_u20(dd(ac, 0.0), &e);
    e += 1;
  } else {
    dd_t w = ddsqrt_d2_d2(ddadd2_d2_d2_d(ddmul_d2_d_d(ac, ac), 1.0));
    lm = oracle_logm_u20(ddadd2_d2_d2_d(w, ac), &e);
  }
  double y = fma((double)e, L2A, lm);
  if (a < TWO_M28) y = a;
  if (!(a <= 0x1.fffffffffffffp1023)) y = isnan(x) ? NAN : INFINITY;
  return canon(copysign(y, x));
}
double oracle_acosh_u35_f64(double x) {
  double xc = (x >= 1 && x <= 0x1.fffffffffffffp1023) ? x : 1.0;
  int e;
  double lm;
  if (xc > 0x1p500) {
    lm = oracle_logm_u20(dd(xc, 0.0), &e);
    e += 1;
  } else {
    dd_t d = ddmul_d2_d2_d2(ddadd2_d2_d_d(xc, -1.0), ddadd2_d2_d_d(xc, 1.0));
    lm = oracle_logm_u20(ddadd2_d2_d2_d(ddsqrt_d2_d2(d), xc), &e);
  }
  double y = fma((double)e, L2A, lm);
  if (xc == 1) y = 0.0;                         /* the DD square root of 0 is not defined */
  if (!(x >= 1 && x <= 0x1.fffffffffffffp1023)) y = x == INFINITY ? INFINITY : NAN;
  return canon(y);
}
double oracle_atanh_u35_f64(double x) {
  double a = fabs(x);
  double ac = a < 1 ? a : 0.5;
  dd_t q = dddiv_d2_d2_d2(ddadd2_d2_d_d(1.0, ac), ddadd2_d2_d_d(1.0, -ac));
  int e;
  double lm = oracle_logm_u20(q, &e);
  double y = 0.5 * fma((double)e, L2A, lm);
  if (a < TWO_M28) y = a;
  if (!(a < 1)) y = a == 1 ? INFINITY : NAN;
  return canon(copysign(y, x));
}

/* ---------------- erf, erfc ----------------
 * erf   |x| < 1: x (C0 + t (C1 + t (c2 + t P(t)))), t = x^2 exact as a DD and
 *       the three leading levels in DD; 1 <= |x| < 6: 1 - erfc(|x|) in DD; +-1 beyond.
 * erfc  |x| < 1: 1 -+ erf(|x|) in DD; 1 <= |x| <= 27.5: F(|x|) e^(-x^2) with
 *       F = erfc(x) e^(x^2) a polynomial about the midpoint of [1,2), [2,4)
 *       or [4,8) (leading two terms in DD) or, from 8 on, G(1/x^2) / (sqrt(pi) x)
 *       with G the asymptotic factor; e^(-x^2) from the DD exp core on the
 *       exact DD x^2 and scaled by 2^k in two steps (subnormal results rounded
 *       once); erfc(-x) = 2 - erfc(x).
 * The u35 erf evaluates the same pieces in double (e^(-x^2) from the
 * residual-carrying reduction and the 12-term e^r - 1 polynomial); the u35
 * erfc runs the u10 algorithm (1 - erf near 1 and the DD argument of the
 * exponential are needed for any bound). */
#define RSQPIH 0x1.20dd750429b6dp-1     /* 1/sqrt(pi) as a DD */
#define RSQPIL 0x1.1ae3a914f6e1fp-57

static const double ERF_H[4] = { ERF_A_HEAD };
static const double ERF_P[11] = { ERF_A_COEFFS };
static const double ERFC_FH[3][4] = { { ERFC_F0_HEAD }, { ERFC_F1_HEAD }, { ERFC_F2_HEAD } };
static const double ERFC_FP[3][22] = { { ERFC_F0_COEFFS }, { ERFC_F1_COEFFS }, { ERFC_F2_COEFFS } };
static const double ERFC_GH[4] = { ERFC_G_HEAD };
static const double ERFC_GP[9] = { ERFC_G_COEFFS };
static const double ERFC_MID[3] = { 1.5, 3.0, 6.0 };

/* erf(a)/a as a DD, 0 <= a < 1: C0 + T (C1 + T (c2 + t P(t))) with T = a^2
 * exact and the three outer levels in DD (1 - erf near a = 1 magnifies the
 * error of erf five-fold) */
static dd_t erf_s(double a) {
  dd_t T = ddmul_d2_d_d(a, a);
  double p = poly_d(T.x, ERF_P + 1, 10);
  dd_t in = ddadd2_d2_d_d(ERF_P[0], T.x * p);
  in = ddadd2_d2_d2_d2(dd(ERF_H[2], ERF_H[3]), ddmul_d2_d2_d2(T, in));
  return ddadd2_d2_d2_d2(dd(ERF_H[0], ERF_H[1]), ddmul_d2_d2_d2(T, in));
}

static int erfc_iv(double a) { return a < 2 ? 0 : (a < 4 ? 1 : 2); }

/* F(a) = erfc(a) e^(a^2) as a DD, 1 <= a <= 27.5 */
static dd_t erfc_F(double a) {
  if (a < 8) {
    int i = erfc_iv(a);
    double u = a - ERFC_MID[i];
    double p = poly_d(u, ERFC_FP[i], 22);
    dd_t in = ddadd2_d2_d2_d(dd(ERFC_FH[i][2], ERFC_FH[i][3]), u * p);
    return ddadd2_d2_d2_d2(dd(ERFC_FH[i][0], ERFC_FH[i][1]), ddmul_d2_d2_d(in, u));
  }
  double w = 1.0 / (a * a);
  double p = poly_d(w, ERFC_GP, 9);
  dd_t in = ddadd2_d2_d2_d(dd(ERFC_GH[2], ERFC_GH[3]), w * p);
  dd_t g = ddadd2_d2_d2_d2(dd(ERFC_GH[0], ERFC_GH[1]), ddmul_d2_d2_d(in, w));
  return dddiv_d2_d2_d2(ddmul_d2_d2_d2(g, dd(RSQPIH, RSQPIL)), dd(a, 0.0));
}

/* erfc(a) = c 2^k with c = F(a) e^(-a^2 - k ln2) as a DD, 1 <= a <= 27.5 */
static dd_t erfc_core(double a, double *k) {
  dd_t Y = ddmul_d2_d_d(a, a);
  dd_t s = oracle_expk_s(dd(-Y.x, -Y.y), k);
  return ddmul_d2_d2_d2(erfc_F(a), ddadd_d2_d_d2(1.0, s));
}

double oracle_erf_u10_f64(double x) {
  double a = fabs(x);
  double y;
  if (a < 1) {
    dd_t e = ddmul_d2_d2_d(erf_s(a), a);
    y = e.x + e.y;
  } else if (a < 6) {
    double k;
    dd_t c = erfc_core(a, &k);
    c = ddscale_d2_d2_d(c, ldexp(1.0, (int)k));
    dd_t r = ddadd2_d2_d_d2(1.0, dd(-c.x, -c.y));
    y = r.x + r.y;
  } else {
    y = 1.0;
  }
  if (isnan(x)) y = NAN;
  return canon(copysign(y, x));
}

double oracle_erfc_u10_f64(double x) {
  double a = fabs(x);
  double y;
  if (a < 1) {
    dd_t e = ddmul_d2_d2_d(erf_s(a), a);
    if (x > 0) e = dd(-e.x, -e.y);
    dd_t r = ddadd2_d2_d_d2(1.0, e);
    y = r.x + r.y;
  } else if (a <= 27.5) {
    double k;
    dd_t c = erfc_core(a, &k);
    if (x > 0) {
      y = oracle_scale2(c.x + c.y, (int)k);
    } else if (a < 8) {
      c = ddscale_d2_d2_d(c, ldexp(1.0, (int)k));
      dd_t r = ddadd2_d2_d_d2(2.0, dd(-c.x, -c.y));
      y = r.x + r.y;
    } else {
      y = 2.0;
    }
  } else {
    y = x > 0 ? 0.0 : 2.0;
  }
  if (isnan(x)) y = NAN;
  return canon(y);
}

double oracle_erf_u35_f64(double x) {
  double a = fabs(x);
  double y;
  if (a < 1) {
    double t = a * a;
    y = a * fma(t, fma(t, poly_d(t, ERF_P, 11), ERF_H[2]), ERF_H[0]);
  } else if (a < 6) {
    int i = erfc_iv(a);
    double u = a - ERFC_MID[i];
    double F = fma(u, fma(u, poly_d(u, ERFC_FP[i], 22), ERFC_FH[i][2]), ERFC_FH[i][0]);
    dd_t Y = ddmul_d2_d_d(a, a);
    double k = rint(-Y.x * R_LN2);
    double r = fma(k, -L2B, fma(k, -L2A, -Y.x)) - Y.y;
    double E = (1.0 + em1_r_u35(r)) * ldexp(1.0, (int)k);
    y = fma(-F, E, 1.0);
  } else {
    y = 1.0;
  }
  if (isnan(x)) y = NAN;
  return canon(copysign(y, x));
}

double oracle_erfc_u35_f64(double x) { return oracle_erfc_u10_f64(x); }

