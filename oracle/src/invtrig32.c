/*
 * FP32 asin, acos, atan and atan2 of the oracle, u10 (float-float where the
 * bound needs it) and u35 (binary32 only).  The paper's FP64 designs
 * (Sections 5.3-5.4) in binary32 with binary32 coefficients.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * asin u = u + u t (c1 + t P(t)), t = u^2, on [0, 1/2]; above it
 * asin a = pi/2 - 2 asin(sqrt((1-a)/2)) with (1-a)/2 exact; acos from the same
 * pieces (pi/2 - asin, 2 asin(..), pi - 2 asin(..)); atan s = s + s t (c1 +
 * t P(t)) on [0, 1], 1/a and pi/2 - atan beyond; atan2 from the atan core
 * on min/max of |x|, |y| (scaled by 2^64 when the smaller is tiny) with the
 * quadrant fix-ups and the C99 Annex F special pairs.
 */
#include "common.h"
#include "coeffs32.h"

#define PIO2HF 0x1.921fb6p+0f
#define PIO2LF (-0x1.777a5cp-25f)
#define PIHF 0x1.921fb6p+1f
#define PILF (-0x1.777a5cp-24f)
#define PIO4F 0x1.921fb6p-1f
#define P3O4F 0x1.2d97c8p+1f

static const float ASIN10[4] = { ASINF_U10_COEFFS };
static const float ASIN35[5] = { ASINF_U35_COEFFS };
static const float ATAN10[9] = { ATANF_U10_COEFFS };
static const float ATAN35[9] = { ATANF_U35_COEFFS };

/* asin of an FF u in [0, 1/2] (u10): u + u t (c1 + t P(t)) */
static ff_t asin_ff(ff_t u) {
  ff_t t = ffsqu_f2_f2(u);
  float p = poly_f(t.x, ASIN10, 4);
  ff_t w = ffadd_f2_f2_f(ff(ASINF_U10_C1H, ASINF_U10_C1L), t.x * p);
  w = ffmul_f2_f2_f2(u, ffmul_f2_f2_f2(t, w));
  return ffadd_f2_f2_f2(u, w);
}
/* sqrt((1 - a)/2) as an FF pair for 1/2 < a <= 1 ((1 - a)/2 is exact) */
static ff_t half_sqrt(float v) { return v > 0 ? ffsqrt_f2_f2(ff(v, 0.0f)) : ff(0.0f, 0.0f); }

static float asin_f(float u) {
  float t = u * u;
  return fmaf(u * t, poly_f(t, ASIN35, 5), u);
}

float oracle_asin_u10_f32(float x) {
  float a = fabsf(x);
  ff_t r;
  if (a <= 0.5f) {
    r = asin_ff(ff(a, 0.0f));
  } else {
    float v = a <= 1.0f ? (1.0f - a) * 0.5f : 0.0f;
    ff_t A = asin_ff(half_sqrt(v));
    r = ffadd2_f2_f2_f2(ff(PIO2HF, PIO2LF), ffscale_f2_f2_f(A, -2.0f));
  }
  float y = r.x + r.y;
  if (!(a <= 1.0f)) y = NAN;
  return canonf(copysignf(y, x));
}
float oracle_asin_u35_f32(float x) {
  float a = fabsf(x), y;
  if (a <= 0.5f) y = asin_f(a);
  else y = fmaf(-2.0f, asin_f(sqrtf(a <= 1.0f ? (1.0f - a) * 0.5f : 0.0f)), PIO2HF);
  if (!(a <= 1.0f)) y = NAN;
  return canonf(copysignf(y, x));
}
float oracle_acos_u10_f32(float x) {
  float a = fabsf(x);
  ff_t r;
  if (a <= 0.5f) {
    ff_t s = asin_ff(ff(a, 0.0f));
    if (x < 0) s = ff(-s.x, -s.y);
    r = ffadd2_f2_f2_f2(ff(PIO2HF, PIO2LF), ff(-s.x, -s.y));
  } else {
    float v = a <= 1.0f ? (1.0f - a) * 0.5f : 0.0f;
    ff_t A = ffscale_f2_f2_f(asin_ff(half_sqrt(v)), 2.0f);
    r = x > 0 ? A : ffadd2_f2_f2_f2(ff(PIHF, PILF), ff(-A.x, -A.y));
  }
  float y = r.x + r.y;
  if (!(a <= 1.0f)) y = NAN;
  return canonf(y);
}
float oracle_acos_u35_f32(float x) {
  float a = fabsf(x), y;
  if (a <= 0.5f) {
    y = PIO2HF - copysignf(asin_f(a), x);
  } else {
    float A = 2.0f * asin_f(sqrtf(a <= 1.0f ? (1.0f - a) * 0.5f : 0.0f));
    y = x > 0 ? A : PIHF - A;
  }
  if (!(a <= 1.0f)) y = NAN;
  return canonf(y);
}

/* atan of an FF s in [0, 1] (u10) */
static ff_t atan_ff(ff_t s) {
  ff_t t = ffsqu_f2_f2(s);
  float p = poly_f(t.x, ATAN10, 9);
  ff_t w = ffadd_f2_f2_f(ff(ATANF_U10_C1H, ATANF_U10_C1L), t.x * p);
  w = ffmul_f2_f2_f2(s, ffmul_f2_f2_f2(t, w));
  return ffadd_f2_f2_f2(s, w);
}
static float atan_f(float s) {
  float t = s * s;
  return fmaf(s * t, poly_f(t, ATAN35, 9), s);
}
float oracle_atan_u10_f32(float x) {
  float a = fabsf(x);
  int big = a > 1.0f;
  ff_t s = big ? (isinf(a) ? ff(0.0f, 0.0f) : ffrec_f2_f(a)) : ff(a, 0.0f);
  ff_t r = atan_ff(s);
  if (big) r = ffadd2_f2_f2_f2(ff(PIO2HF, PIO2LF), ff(-r.x, -r.y));
  float y = r.x + r.y;
  if (isnan(x)) y = NAN;
  return canonf(copysignf(y, x));
}
float oracle_atan_u35_f32(float x) {
  float a = fabsf(x);
  float y = a > 1.0f ? PIO2HF - atan_f(1.0f / a) : atan_f(a);
  if (isnan(x)) y = NAN;
  return canonf(copysignf(y, x));
}

/* atan2(y, x) in C order: the ordinate first */
static float atan2f_core(float y, float x, int u10) {
  float ay = fabsf(y), ax = fabsf(x);
  float mn = ay < ax ? ay : ax, mx = ay < ax ? ax : ay;
  /* the FF division's remainder must not underflow: tiny operands are
   * scaled by 2^64 together; a ratio below 2^-120 is one rounded division */
  int plain = mn < 0x1p-60f && mx >= 0x1p60f;
  if (mx < 0x1p-60f || (mn < 0x1p-60f && mx < 0x1p60f)) { mn *= 0x1p64f; mx *= 0x1p64f; }
  float r;
  if (u10) {
    ff_t s = plain ? ff(mn / mx, 0.0f) : ffdiv_f2_f2_f2(ff(mn, 0.0f), ff(mx, 0.0f));
    ff_t t = atan_ff(s);
    if (ay > ax) t = ffadd2_f2_f2_f2(ff(PIO2HF, PIO2LF), ff(-t.x, -t.y));
    if (signbit(x)) t = ffadd2_f2_f2_f2(ff(PIHF, PILF), ff(-t.x, -t.y));
    r = t.x + t.y;
  } else {
    float t = atan_f(mn / mx);
    if (ay > ax) t = PIO2HF - t;
    if (signbit(x)) t = PIHF - t;
    r = t;
  }
  /* C99 Annex F special pairs */
  if (ay == 0) r = signbit(x) ? PIHF : 0.0f;
  else if (ax == 0 || (isinf(ay) && !isinf(ax))) r = PIO2HF;
  else if (isinf(ax)) r = isinf(ay) ? (signbit(x) ? 3.0f * PIO4F : PIO4F) : (signbit(x) ? PIHF : 0.0f);
  r = copysignf(r, y);
  if (isnan(x) || isnan(y)) r = NAN;
  return canonf(r);
}
float oracle_atan2_u10_f32(float y, float x) { return atan2f_core(y, x, 1); }
float oracle_atan2_u35_f32(float y, float x) { return atan2f_core(y, x, 0); }
