/*
 * The remaining C99 real functions of the oracle, binary64 and binary32.
 *
 * Exact functions (their names carry no accuracy tag): fabs, copysign, fmax,
 * fmin, fdim, trunc, floor, ceil, round, rint, nextafter, logb, ilogb, ldexp,
 * frexp and modf.  Each is written out from its definition in C99 (7.12 and
 * Annex F) on the fields of the IEEE encoding (sign, biased exponent,
 * significand), with integer rounding where a result is rounded (rint,
 * round, ldexp into the subnormal range).  Every NaN result is the canonical
 * quiet NaN, fabs and copysign included (as everywhere in the library).
 * Choices C99 leaves open: fmax(+0, -0) = +0 and fmin(+0, -0) = -0;
 * ilogb(0) = INT_MIN, ilogb(NaN) = INT_MAX; frexp(inf or NaN) stores 0.
 *
 * Approximated functions, each in a 0.5-ULP and a 3.5-ULP form:
 *   sqrt   the IEEE square root, correctly rounded (both forms)
 *   hypot  |x| and |y| scaled by the exponent of the larger (exactly), the
 *          sum of squares in DD (FF) arithmetic and its DD (FF) square root
 *          for u05; one fma and a square root for u35
 *   sinpi, cospi  the exact reduction x = q/2 + s, |s| <= 1/4, q = rint(2x),
 *          then sin(pi s) or cos(pi s) by the quadrant q mod 4; each a single
 *          polynomial in t = s^2 (Section 5's scheme), its leading terms in
 *          DD (FF) arithmetic for u05 and plain for u35
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#include <limits.h>
#include "oracle.h"
#include "coeffs32.h"
#include "coeffs64.h"

/* ---------------- the IEEE fields, for either format ----------------
 * mant = stored significand bits (52 / 23), ebits = exponent bits (11 / 8) */
typedef struct { int mant, ebits; } fmt_t;
static const fmt_t F64 = { 52, 11 }, F32 = { 23, 8 };

static uint64_t sgn_bit(fmt_t f) { return 1ULL << (f.mant + f.ebits); }
static int bias_of(fmt_t f) { return (1 << (f.ebits - 1)) - 1; }
static int emax_field(fmt_t f) { return (1 << f.ebits) - 1; }
static uint64_t fracm(fmt_t f) { return (1ULL << f.mant) - 1; }
static int bexp(uint64_t b, fmt_t f) { return (int)((b >> f.mant) & (uint64_t)emax_field(f)); }
static int is_nan_b(uint64_t b, fmt_t f) { return bexp(b, f) == emax_field(f) && (b & fracm(f)) != 0; }
static int is_inf_b(uint64_t b, fmt_t f) { return bexp(b, f) == emax_field(f) && (b & fracm(f)) == 0; }
static int is_zero_b(uint64_t b, fmt_t f) { return (b & ~sgn_bit(f)) == 0; }
static int msb64(uint64_t v) { return 63 - __builtin_clzll(v); }

static uint64_t b64(double d) { return dbits(d); }
static double d64(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t b32(float x) { return fbits(x); }
static float f32(uint64_t b) { uint32_t u = (uint32_t)b; float x; memcpy(&x, &u, 4); return x; }
static uint64_t qnan_b(fmt_t f) { return ((uint64_t)emax_field(f) << f.mant) | (1ULL << (f.mant - 1)); }

/* the unbiased exponent of a finite non-zero encoding: x = 1.f 2^e */
static int ilogb_fin(uint64_t b, fmt_t f) {
  int E = bexp(b, f);
  if (E != 0) return E - bias_of(f);
  return msb64(b & fracm(f)) - f.mant + 1 - bias_of(f);
}

/* the encoding of sign | q for an integer 0 <= q < 2^(mant+2) (exact) */
static uint64_t from_int(uint64_t sign, uint64_t q, fmt_t f) {
  if (q == 0) return sign;
  int p = msb64(q);
  uint64_t sig = p <= f.mant ? q << (f.mant - p) : q >> (p - f.mant);
  return sign | ((uint64_t)(p + bias_of(f)) << f.mant) | (sig & fracm(f));
}

/* trunc: clear the fraction bits below the binary point */
static uint64_t trunc_b(uint64_t b, fmt_t f) {
  int E = bexp(b, f), e = E - bias_of(f);
  if (E == emax_field(f) || e >= f.mant) return b;
  if (e < 0) return b & sgn_bit(f);
  return b & ~(fracm(f) >> e);
}

/* rint (ties to even, away = 0) and round (ties away from zero, away = 1):
 * the integer quotient and remainder of the significand */
static uint64_t rnd_b(uint64_t b, fmt_t f, int away) {
  int E = bexp(b, f), e = E - bias_of(f);
  uint64_t sign = b & sgn_bit(f);
  if (E == emax_field(f) || e >= f.mant) return b;
  if (e < -1) return sign;                        /* |x| < 1/2 */
  uint64_t M = (b & fracm(f)) | (1ULL << f.mant);
  int s = f.mant - e;                             /* 1 .. mant + 1 */
  uint64_t q = M >> s, r = M & ((1ULL << s) - 1), half = 1ULL << (s - 1);
  int up = away ? r >= half : (r > half || (r == half && (q & 1)));
  return from_int(sign, q + (uint64_t)up, f);
}

/* ldexp: x 2^n rounded once (ties to even), through the integer significand */
static uint64_t ldexp_b(uint64_t b, long n, fmt_t f) {
  uint64_t sign = b & sgn_bit(f);
  if (is_nan_b(b, f)) return qnan_b(f);
  if (is_inf_b(b, f) || is_zero_b(b, f)) return b;
  if (n > 100000) n = 100000;
  if (n < -100000) n = -100000;
  int E = bexp(b, f);
  uint64_t M = E ? (b & fracm(f)) | (1ULL << f.mant) : b & fracm(f);
  long e = (E ? E : 1) - bias_of(f) - f.mant;     /* x = M 2^e */
  int lz = f.mant - msb64(M);                     /* normalise M to mant + 1 bits */
  M <<= lz;
  e = e - lz + n;
  long top = e + f.mant;                          /* exponent of the leading bit */
  int emin = 1 - bias_of(f);
  if (top > bias_of(f)) return sign | ((uint64_t)emax_field(f) << f.mant);   /* overflow: inf */
  if (top >= emin) return sign | ((uint64_t)(top + bias_of(f)) << f.mant) | (M & fracm(f));
  long s = (long)(emin - f.mant) - e;             /* > 0 bits below the subnormal grid */
  if (s > f.mant + 2) return sign;                /* below half the least subnormal */
  uint64_t q = M >> s, r = M & ((1ULL << s) - 1), half = 1ULL << (s - 1);
  q += (r > half || (r == half && (q & 1)));
  return sign | q;                                /* q = 2^mant carries into the least normal */
}

/* frexp: x = m 2^k with |m| in [1/2, 1) */
static uint64_t frexp_b(uint64_t b, int32_t *k, fmt_t f) {
  *k = 0;
  if (is_nan_b(b, f)) return qnan_b(f);
  if (is_inf_b(b, f) || is_zero_b(b, f)) return b;
  int e = ilogb_fin(b, f);
  *k = e + 1;
  return ldexp_b(b, -(long)(e + 1), f);           /* exact: the result is normal */
}

static int32_t ilogb_b(uint64_t b, fmt_t f) {
  if (is_nan_b(b, f)) return INT_MAX;
  if (is_inf_b(b, f)) return INT_MAX;
  if (is_zero_b(b, f)) return INT_MIN;
  return ilogb_fin(b, f);
}

/* ---------------- binary64 exact functions ---------------- */
double oracle_fabs_f64(double x) { return canon(d64(b64(x) & ~sgn_bit(F64))); }
double oracle_copysign_f64(double x, double y) {
  return canon(d64((b64(x) & ~sgn_bit(F64)) | (b64(y) & sgn_bit(F64))));
}
double oracle_trunc_f64(double x) { return canon(d64(trunc_b(b64(x), F64))); }
double oracle_floor_f64(double x) {
  double t = d64(trunc_b(b64(x), F64));
  if (isnan(x)) return canon_nan();
  return (t != x && x < 0) ? t - 1.0 : t;         /* |t| < 2^52: exact */
}
double oracle_ceil_f64(double x) {
  double t = d64(trunc_b(b64(x), F64));
  if (isnan(x)) return canon_nan();
  return (t != x && x > 0) ? t + 1.0 : t;
}
double oracle_rint_f64(double x) { return canon(d64(rnd_b(b64(x), F64, 0))); }
double oracle_round_f64(double x) { return canon(d64(rnd_b(b64(x), F64, 1))); }
double oracle_logb_f64(double x) {
  uint64_t b = b64(x);
  if (is_nan_b(b, F64)) return canon_nan();
  if (is_inf_b(b, F64)) return INFINITY;
  if (is_zero_b(b, F64)) return -INFINITY;
  return (double)ilogb_fin(b, F64);
}
int32_t oracle_ilogb_f64(double x) { return ilogb_b(b64(x), F64); }
double oracle_ldexp_f64(double x, int32_t n) { return d64(ldexp_b(b64(x), n, F64)); }
double oracle_frexp_f64(double x, int32_t *k) { return d64(frexp_b(b64(x), k, F64)); }
void oracle_modf_f64(double x, double *frac, double *ip) {
  if (isnan(x)) { *frac = *ip = canon_nan(); return; }
  double t = d64(trunc_b(b64(x), F64));
  double r = isinf(x) ? 0.0 : x - t;              /* exact */
  *ip = t;
  *frac = oracle_copysign_f64(r, x);
}
double oracle_fmax_f64(double x, double y) {
  if (isnan(x)) return canon(y);
  if (isnan(y)) return x;
  if (x == y) return signbit(x) ? y : x;          /* +0 over -0 */
  return x > y ? x : y;
}
double oracle_fmin_f64(double x, double y) {
  if (isnan(x)) return canon(y);
  if (isnan(y)) return x;
  if (x == y) return signbit(x) ? x : y;          /* -0 over +0 */
  return x < y ? x : y;
}
double oracle_fdim_f64(double x, double y) {
  if (isnan(x) || isnan(y)) return canon_nan();
  return x > y ? x - y : 0.0;
}
double oracle_nextafter_f64(double x, double y) {
  if (isnan(x) || isnan(y)) return canon_nan();
  if (x == y) return y;
  if (x == 0) return d64((b64(y) & sgn_bit(F64)) | 1);
  uint64_t b = b64(x);
  return d64(((x < y) == (x > 0)) ? b + 1 : b - 1);
}

/* ---------------- binary32 exact functions ---------------- */
float oracle_fabs_f32(float x) { return canonf(f32(b32(x) & ~sgn_bit(F32))); }
float oracle_copysign_f32(float x, float y) {
  return canonf(f32((b32(x) & ~sgn_bit(F32)) | (b32(y) & sgn_bit(F32))));
}
float oracle_trunc_f32(float x) { return canonf(f32(trunc_b(b32(x), F32))); }
float oracle_floor_f32(float x) {
  float t = f32(trunc_b(b32(x), F32));
  if (isnan(x)) return canon_nanf();
  return (t != x && x < 0) ? t - 1.0f : t;
}
float oracle_ceil_f32(float x) {
  float t = f32(trunc_b(b32(x), F32));
  if (isnan(x)) return canon_nanf();
  return (t != x && x > 0) ? t + 1.0f : t;
}
float oracle_rint_f32(float x) { return canonf(f32(rnd_b(b32(x), F32, 0))); }
float oracle_round_f32(float x) { return canonf(f32(rnd_b(b32(x), F32, 1))); }
float oracle_logb_f32(float x) {
  uint64_t b = b32(x);
  if (is_nan_b(b, F32)) return canon_nanf();
  if (is_inf_b(b, F32)) return INFINITY;
  if (is_zero_b(b, F32)) return -INFINITY;
  return (float)ilogb_fin(b, F32);
}
int32_t oracle_ilogb_f32(float x) { return ilogb_b(b32(x), F32); }
float oracle_ldexp_f32(float x, int32_t n) { return f32(ldexp_b(b32(x), n, F32)); }
float oracle_frexp_f32(float x, int32_t *k) { return f32(frexp_b(b32(x), k, F32)); }
void oracle_modf_f32(float x, float *frac, float *ip) {
  if (isnan(x)) { *frac = *ip = canon_nanf(); return; }
  float t = f32(trunc_b(b32(x), F32));
  float r = isinf(x) ? 0.0f : x - t;
  *ip = t;
  *frac = oracle_copysign_f32(r, x);
}
float oracle_fmax_f32(float x, float y) {
  if (isnan(x)) return canonf(y);
  if (isnan(y)) return x;
  if (x == y) return signbit(x) ? y : x;
  return x > y ? x : y;
}
float oracle_fmin_f32(float x, float y) {
  if (isnan(x)) return canonf(y);
  if (isnan(y)) return x;
  if (x == y) return signbit(x) ? x : y;
  return x < y ? x : y;
}
float oracle_fdim_f32(float x, float y) {
  if (isnan(x) || isnan(y)) return canon_nanf();
  return x > y ? x - y : 0.0f;
}
float oracle_nextafter_f32(float x, float y) {
  if (isnan(x) || isnan(y)) return canon_nanf();
  if (x == y) return y;
  if (x == 0) return f32((b32(y) & sgn_bit(F32)) | 1);
  uint64_t b = b32(x);
  return f32(((x < y) == (x > 0)) ? b + 1 : b - 1);
}

/* ---------------- sqrt ---------------- */
double oracle_sqrt_u05_f64(double x) { return canon(sqrt(x)); }
double oracle_sqrt_u35_f64(double x) { return canon(sqrt(x)); }
float oracle_sqrt_u05_f32(float x) { return canonf(sqrtf(x)); }
float oracle_sqrt_u35_f32(float x) { return canonf(sqrtf(x)); }

/* ---------------- hypot ----------------
 * Annex F: an infinite operand gives +inf even when the other is a NaN.
 * With a = max(|x|, |y|) = 1.f 2^e, a 2^-e is exact and b 2^-e <= a 2^-e. */
static double hypot64(double x, double y, int u05) {
  double a = fabs(x), b = fabs(y);
  if (isinf(x) || isinf(y)) return INFINITY;
  if (isnan(x) || isnan(y)) return canon_nan();
  if (a < b) { double t = a; a = b; b = t; }
  if (b == 0) return a;
  int e = ilogb(a);
  double as = ldexp(a, -e), bs = ldexp(b, -e);
  double r;
  if (u05) {
    dd_t s = ddadd_d2_d2_d2(ddmul_d2_d_d(as, as), ddmul_d2_d_d(bs, bs));
    dd_t q = ddsqrt_d2_d2(s);
    r = q.x + q.y;
  } else {
    r = sqrt(fma(as, as, bs * bs));
  }
  return ldexp(r, e);
}
double oracle_hypot_u05_f64(double x, double y) { return hypot64(x, y, 1); }
double oracle_hypot_u35_f64(double x, double y) { return hypot64(x, y, 0); }

static float hypot32(float x, float y, int u05) {
  float a = fabsf(x), b = fabsf(y);
  if (isinf(x) || isinf(y)) return INFINITY;
  if (isnan(x) || isnan(y)) return canon_nanf();
  if (a < b) { float t = a; a = b; b = t; }
  if (b == 0) return a;
  int e = ilogbf(a);
  float as = ldexpf(a, -e), bs = ldexpf(b, -e);
  float r;
  if (u05) {
    ff_t s = ffadd_f2_f2_f2(ffmul_f2_f_f(as, as), ffmul_f2_f_f(bs, bs));
    ff_t q = ffsqrt_f2_f2(s);
    r = q.x + q.y;
  } else {
    r = sqrtf(fmaf(as, as, bs * bs));
  }
  return ldexpf(r, e);
}
float oracle_hypot_u05_f32(float x, float y) { return hypot32(x, y, 1); }
float oracle_hypot_u35_f32(float x, float y) { return hypot32(x, y, 0); }

/* ---------------- sinpi, cospi ----------------
 * sin(pi s) = s g(t) and cos(pi s) = 1 + t f(t), t = s^2, |s| <= 1/4, with
 * g and f of eight coefficients each.  Both take one shape, so that an
 * element's quadrant only selects coefficients (Section 5's branch-free
 * evaluation): P = k0 + t (k1 + t (k2 + t p(t))), p the plain polynomial of
 * the five highest coefficients (three in binary32, cos padded with a zero),
 * then sin(pi s) = s P and cos(pi s) = 1 + t P.  In the 0.5-ULP forms k0 and
 * k1 are DD (FF) pairs and the three outer Horner steps are DD (FF) steps,
 * so that the rounding of p is damped by t^3; for |s| < 2^-500 (2^-100) the
 * sine is evaluated on s 2^200 (s 2^80) and scaled back, so that the DD (FF)
 * tails stay representable (the scaled argument stays below 2^-300 (2^-20),
 * where sin(pi s) is pi s to far below an ulp).  The 3.5-ULP forms take the heads and plain
 * Horner steps. */
static const double SPI_H[4] = { C99_SINPI_HEAD };     /* g: k0 (hi, lo), k1 (hi, lo) */
static const double SPI_P[6] = { C99_SINPI_COEFFS };   /* g: k2, then p */
static const double CPI_H[2] = { C99_COSPI_HEAD };     /* f: k0 (hi, lo) */
static const double CPI_P[7] = { C99_COSPI_COEFFS };   /* f: k1, k2, then p */

typedef struct { dd_t k0, k1; double k2; const double *p; } pik_t;
static pik_t pi_coeffs(int cosine) {
  pik_t c;
  if (cosine) { c.k0 = dd(CPI_H[0], CPI_H[1]); c.k1 = dd(CPI_P[0], 0.0); c.k2 = CPI_P[1]; c.p = CPI_P + 2; }
  else { c.k0 = dd(SPI_H[0], SPI_H[1]); c.k1 = dd(SPI_H[2], SPI_H[3]); c.k2 = SPI_P[0]; c.p = SPI_P + 1; }
  return c;
}

/* x = q/2 + s exactly, with q = rint(2x) and o = q mod 4; |x| >= 2^53 is an
 * even integer (o = 0, s = 0) */
static double reduce_pi(double x, int *o) {
  if (fabs(x) >= 0x1p53) { *o = 0; return 0.0; }
  double q = rint(x + x);
  *o = low2_of_integral(q);
  return x - 0.5 * q;
}

static double sincospi64(double x, int cosine, int u05) {
  int o;
  if (isnan(x) || isinf(x)) return canon_nan();
  double s = reduce_pi(x, &o);
  o = (o + cosine) & 3;                       /* cos(pi x) = sin(pi (x + 1/2)) */
  int c = o & 1;                              /* the cosine polynomial of s */
  pik_t k = pi_coeffs(c);
  double v;
  if (u05) {
    int tiny = !c && fabs(s) < 0x1p-500;
    if (tiny) s *= 0x1p200;
    dd_t t = ddmul_d2_d_d(s, s);
    double p = poly_d(t.x, k.p, 5);
    dd_t P = ddadd2_d2_d_d(k.k2, t.x * p);
    P = ddadd2_d2_d2_d2(k.k1, ddmul_d2_d2_d2(t, P));
    P = ddadd2_d2_d2_d2(k.k0, ddmul_d2_d2_d2(t, P));
    dd_t r = c ? ddadd2_d2_d_d2(1.0, ddmul_d2_d2_d2(t, P)) : ddmul_d2_d2_d(P, s);
    v = r.x + r.y;
    if (tiny) v *= 0x1p-200;
  } else {
    double t = s * s;
    double p = poly_d(t, k.p, 5);
    double P = fma(t, fma(t, fma(t, p, k.k2), k.k1.x), k.k0.x);
    v = c ? fma(t, P, 1.0) : s * P;
  }
  if (o & 2) v = -v;
  /* zero results: sinpi(n) = +-0 with the sign of n, cospi(n + 1/2) = +0 */
  if (v == 0) v = cosine ? 0.0 : copysign(0.0, x);
  return v;
}
double oracle_sinpi_u05_f64(double x) { return sincospi64(x, 0, 1); }
double oracle_sinpi_u35_f64(double x) { return sincospi64(x, 0, 0); }
double oracle_cospi_u05_f64(double x) { return sincospi64(x, 1, 1); }
double oracle_cospi_u35_f64(double x) { return sincospi64(x, 1, 0); }

static const float SPIF_H[4] = { C99_SINPIF_HEAD };
static const float SPIF_P[4] = { C99_SINPIF_COEFFS };
static const float CPIF_H[2] = { C99_COSPIF_HEAD };
static const float CPIF_P[5] = { C99_COSPIF_COEFFS, 0.0f };

typedef struct { ff_t k0, k1; float k2; const float *p; } pikf_t;
static pikf_t pi_coeffsf(int cosine) {
  pikf_t c;
  if (cosine) { c.k0 = ff(CPIF_H[0], CPIF_H[1]); c.k1 = ff(CPIF_P[0], 0.0f); c.k2 = CPIF_P[1]; c.p = CPIF_P + 2; }
  else { c.k0 = ff(SPIF_H[0], SPIF_H[1]); c.k1 = ff(SPIF_H[2], SPIF_H[3]); c.k2 = SPIF_P[0]; c.p = SPIF_P + 1; }
  return c;
}
static float reduce_pif(float x, int *o) {
  if (fabsf(x) >= 0x1p24f) { *o = 0; return 0.0f; }
  float q = rintf(x + x);
  *o = low2_of_integralf(q);
  return x - 0.5f * q;
}
static float sincospi32(float x, int cosine, int u05) {
  int o;
  if (isnan(x) || isinf(x)) return canon_nanf();
  float s = reduce_pif(x, &o);
  o = (o + cosine) & 3;
  int c = o & 1;
  pikf_t k = pi_coeffsf(c);
  float v;
  if (u05) {
    int tiny = !c && fabsf(s) < 0x1p-100f;
    if (tiny) s *= 0x1p80f;
    ff_t t = ffmul_f2_f_f(s, s);
    float p = poly_f(t.x, k.p, 3);
    ff_t P = ffadd2_f2_f_f(k.k2, t.x * p);
    P = ffadd2_f2_f2_f2(k.k1, ffmul_f2_f2_f2(t, P));
    P = ffadd2_f2_f2_f2(k.k0, ffmul_f2_f2_f2(t, P));
    ff_t r = c ? ffadd2_f2_f_f2(1.0f, ffmul_f2_f2_f2(t, P)) : ffmul_f2_f2_f(P, s);
    v = r.x + r.y;
    if (tiny) v *= 0x1p-80f;
  } else {
    float t = s * s;
    float p = poly_f(t, k.p, 3);
    float P = fmaf(t, fmaf(t, fmaf(t, p, k.k2), k.k1.x), k.k0.x);
    v = c ? fmaf(t, P, 1.0f) : s * P;
  }
  if (o & 2) v = -v;
  if (v == 0) v = cosine ? 0.0f : copysignf(0.0f, x);
  return v;
}
float oracle_sinpi_u05_f32(float x) { return sincospi32(x, 0, 1); }
float oracle_sinpi_u35_f32(float x) { return sincospi32(x, 0, 0); }
float oracle_cospi_u05_f32(float x) { return sincospi32(x, 1, 1); }
float oracle_cospi_u35_f32(float x) { return sincospi32(x, 1, 0); }
