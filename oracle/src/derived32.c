/*
 * FP32 functions of the oracle built on the binary32 exp/log cores:
 * exp2, exp10, expm1, log2, log10, sinh, cosh, asinh, acosh, atanh, pow,
 * cbrt and erfc, u10 and u35.  The paper describes the FP64 functions; these
 * mirror the FP64 designs of derived64.c in float-float (FF) arithmetic with
 * binary32 coefficients and no FP64 anywhere.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * Where no cheaper binary32 form keeps 3.5 ULP (expm1, sinh, cosh, the
 * inverse hyperbolics, pow, erfc), the u35 entry point runs the u10
 * algorithm.
 */
#include "common.h"
#include "coeffs32.h"
#include "explog32.h"

#define R_LN2F 0x1.715476p0f
#define L2AF 0x1.62e430p-1f
#define L2BF (-0x1.05c610p-29f)
#define L2HF 0x1.62e400p-1f
#define L2LF 0x1.7f7d1cp-20f
#define LN10HF 0x1.26bb1cp+1f
#define LN10LF (-0x1.12aabap-25f)
#define RL2HF 0x1.715476p+0f
#define RL2LF 0x1.4ae0c0p-26f
#define RL10HF 0x1.bcb7b2p-2f
#define RL10LF (-0x1.5b235ep-27f)
#define L10AF 0x1.344136p-2f
#define L10BF (-0x1.ec10c0p-27f)
#define LG2HF 0x1.344000p-2f
#define LG2LF 0x1.3509f8p-18f
#define LOG2_10F 0x1.a934f0p+1f
#define THIRDF 0x1.555556p-2f
#define FLT_MAXF 0x1.fffffep127f

static const float EXPF_U35[5] = { EXPF_U35_COEFFS };
static const float CBRTF[4] = { CBRTF_COEFFS };

/* ---------------- exp2, exp10 ---------------- */
static float expf_out(float x, float y, float lim) {
  if (!(fabsf(x) <= lim)) y = x > 0 ? INFINITY : (x < 0 ? 0.0f : NAN);
  return canonf(y);
}
float oracle_exp2_u10_f32(float x) {
  float xc = fabsf(x) <= 160.0f ? x : 0.0f;
  float k = rintf(xc);
  ff_t t = ffmul_f2_f2_f(ff(L2AF, L2BF), xc - k);
  return expf_out(x, oracle_expf_tail_u10(t.x, t.y, k), 160.0f);
}
float oracle_exp2_u35_f32(float x) {
  float xc = fabsf(x) <= 160.0f ? x : 0.0f;
  float k = rintf(xc);
  float t = (xc - k) * L2AF;
  float v = fmaf(t * t, poly_f(t, EXPF_U35, 5), t);
  return expf_out(x, oracle_scale2f(1.0f + v, (int)k), 160.0f);
}
float oracle_exp10_u10_f32(float x) {
  float xc = fabsf(x) <= 50.0f ? x : 0.0f;
  float k = rintf(xc * LOG2_10F);
  float h = fmaf(k, -L10AF, xc);
  float r = fmaf(k, -L10BF, h);
  float rl = fmaf(k, -L10BF, h - r);
  ff_t t = ffmul_f2_f2_f2(ff(r, rl), ff(LN10HF, LN10LF));
  return expf_out(x, oracle_expf_tail_u10(t.x, t.y, k), 50.0f);
}
float oracle_exp10_u35_f32(float x) {
  float xc = fabsf(x) <= 50.0f ? x : 0.0f;
  float k = rintf(xc * LOG2_10F);
  float t = fmaf(k, -L10BF, fmaf(k, -L10AF, xc)) * LN10HF;
  float v = fmaf(t * t, poly_f(t, EXPF_U35, 5), t);
  return expf_out(x, oracle_scale2f(1.0f + v, (int)k), 50.0f);
}

/* ---------------- expm1 ---------------- */
/* e^a - 1 as an FF pair for -18 < a <= 40 (2^k - 1 exact as an FF pair) */
static ff_t em1f(float a) {
  float k;
  ff_t s = oracle_expm1f_s(a, &k);
  float p = ldexpf(1.0f, (int)k);
  return ffadd2_f2_f2_f2(ffadd2_f2_f_f(p, -1.0f), ffscale_f2_f2_f(s, p));
}
float oracle_expm1_u10_f32(float x) {
  float xc = (x > -18.0f && x < 89.0f) ? x : 0.0f;
  float k;
  ff_t s = oracle_expm1f_s(xc, &k);
  float y;
  if (k > 100) {
    ff_t e = ffadd_f2_f_f2(1.0f, s);
    y = oracle_scale2f(e.x + e.y, (int)k);
  } else {
    float p = ldexpf(1.0f, (int)k);
    ff_t r = ffadd2_f2_f2_f2(ffadd2_f2_f_f(p, -1.0f), ffscale_f2_f2_f(s, p));
    y = r.x + r.y;
  }
  if (x == 0) y = x;
  if (!(x > -18.0f && x < 89.0f)) y = x >= 89.0f ? INFINITY : (x <= -18.0f ? -1.0f : NAN);
  return canonf(y);
}
float oracle_expm1_u35_f32(float x) { return oracle_expm1_u10_f32(x); }

/* ---------------- log2, log10 ---------------- */
static float logf_out(float x, float y) {
  if (x == 0) return -INFINITY;
  if (x < 0 || isnan(x)) return canonf(NAN);
  if (isinf(x)) return INFINITY;
  return canonf(y);
}
float oracle_log2_u10_f32(float x) {
  float a = (x > 0 && x <= FLT_MAXF) ? x : 1.0f;
  int e;
  ff_t lm = oracle_logmf_u10(ff(a, 0.0f), &e);
  ff_t p = ffmul_f2_f2_f2(lm, ff(RL2HF, RL2LF));
  ff_t r = ffadd2_f2_f_f2((float)e, p);
  return logf_out(x, r.x + r.y);
}
float oracle_log2_u35_f32(float x) {
  float a = (x > 0 && x <= FLT_MAXF) ? x : 1.0f;
  int e;
  ff_t lm = oracle_logmf_u10(ff(a, 0.0f), &e);
  return logf_out(x, fmaf(lm.x + lm.y, RL2HF, (float)e));
}
float oracle_log10_u10_f32(float x) {
  float a = (x > 0 && x <= FLT_MAXF) ? x : 1.0f;
  int e;
  ff_t lm = oracle_logmf_u10(ff(a, 0.0f), &e);
  ff_t p = ffmul_f2_f2_f2(lm, ff(RL10HF, RL10LF));
  float ed = (float)e;
  ff_t r = ffadd2_f2_f2_f2(ff(ed * LG2HF, ed * LG2LF), p);
  return logf_out(x, r.x + r.y);
}
float oracle_log10_u35_f32(float x) {
  float a = (x > 0 && x <= FLT_MAXF) ? x : 1.0f;
  int e;
  ff_t lm = oracle_logmf_u10(ff(a, 0.0f), &e);
  return logf_out(x, fmaf((float)e, L10AF, (lm.x + lm.y) * RL10HF));
}

/* ---------------- sinh, cosh ---------------- */
/* e^a / 2 for 12 < a <= 89.5: e^(a - ln2) with the argument an FF pair */
static float exph_big(float a) {
  float k;
  ff_t o = oracle_expf_parts(ffadd2_f2_f_f2(a, ff(-L2AF, -L2BF)), &k);
  return oracle_scale2f(o.x + o.y, (int)k);
}
float oracle_sinh_u10_f32(float x) {
  float a = fabsf(x);
  float ac = a <= 89.5f ? a : 0.0f;
  float y;
  if (ac > 12.0f) {
    y = exph_big(ac);
  } else {
    ff_t em = em1f(ac);
    ff_t f = ffdiv_f2_f2_f2(em, ffadd2_f2_f_f2(1.0f, em));
    ff_t h = ffadd2_f2_f2_f2(em, f);
    y = 0.5f * (h.x + h.y);
  }
  if (a < 0x1p-12f) y = a;
  if (!(a <= 89.5f)) y = isnan(x) ? NAN : INFINITY;
  return canonf(copysignf(y, x));
}
float oracle_cosh_u10_f32(float x) {
  float a = fabsf(x);
  float ac = a <= 89.5f ? a : 0.0f;
  float y;
  if (ac > 12.0f) {
    y = exph_big(ac);
  } else {
    ff_t E = ffadd2_f2_f_f2(1.0f, em1f(ac));
    ff_t h = ffadd_f2_f2_f2(E, ffrec_f2_f2(E));
    y = 0.5f * (h.x + h.y);
  }
  if (!(a <= 89.5f)) y = isnan(x) ? NAN : INFINITY;
  return canonf(y);
}
float oracle_sinh_u35_f32(float x) { return oracle_sinh_u10_f32(x); }
float oracle_cosh_u35_f32(float x) { return oracle_cosh_u10_f32(x); }

/* ---------------- asinh, acosh, atanh ---------------- */
float oracle_asinh_u10_f32(float x) {
  float a = fabsf(x);
  float ac = a <= FLT_MAXF ? a : 1.0f;
  ff_t r;
  if (ac > 0x1p60f) {
    r = ffadd2_f2_f2_f2(oracle_logf_ff(ff(ac, 0.0f)), ff(L2AF, L2BF));
  } else {
    ff_t w = ffsqrt_f2_f2(ffadd2_f2_f2_f(ffmul_f2_f_f(ac, ac), 1.0f));
    r = oracle_logf_ff(ffadd2_f2_f2_f(w, ac));
  }
  float y = r.x + r.y;
  if (a < 0x1p-12f) y = a;
  if (!(a <= FLT_MAXF)) y = isnan(x) ? NAN : INFINITY;
  return canonf(copysignf(y, x));
}
float oracle_acosh_u10_f32(float x) {
  float xc = (x >= 1.0f && x <= FLT_MAXF) ? x : 1.0f;
  ff_t r;
  if (xc > 0x1p60f) {
    r = ffadd2_f2_f2_f2(oracle_logf_ff(ff(xc, 0.0f)), ff(L2AF, L2BF));
  } else {
    ff_t d = ffmul_f2_f2_f2(ffadd2_f2_f_f(xc, -1.0f), ffadd2_f2_f_f(xc, 1.0f));
    r = oracle_logf_ff(ffadd2_f2_f2_f(ffsqrt_f2_f2(d), xc));
  }
  float y = r.x + r.y;
  if (xc == 1.0f) y = 0.0f;
  if (!(x >= 1.0f && x <= FLT_MAXF)) y = x == INFINITY ? INFINITY : NAN;
  return canonf(y);
}
float oracle_atanh_u10_f32(float x) {
  float a = fabsf(x);
  float ac = a < 1.0f ? a : 0.5f;
  ff_t q = ffdiv_f2_f2_f2(ffadd2_f2_f_f(1.0f, ac), ffadd2_f2_f_f(1.0f, -ac));
  ff_t r = oracle_logf_ff(q);
  float y = 0.5f * (r.x + r.y);
  if (a < 0x1p-12f) y = a;
  if (!(a < 1.0f)) y = a == 1.0f ? INFINITY : NAN;
  return canonf(copysignf(y, x));
}
/* 3.5-ULP forms: the same FF arguments, their logarithm in binary32 with z
 * corrected once (oracle_logmf_u20) and e ln 2 added by one fma; above 2^60
 * log(2x) = (e + 1) ln 2 + log m */
float oracle_asinh_u35_f32(float x) {
  float a = fabsf(x);
  float ac = a <= FLT_MAXF ? a : 1.0f;
  int e;
  float lm;
  if (ac > 0x1p60f) {
    lm = oracle_logmf_u20(ff(ac, 0.0f), &e);
    e += 1;
  } else {
    ff_t w = ffsqrt_f2_f2(ffadd2_f2_f2_f(ffmul_f2_f_f(ac, ac), 1.0f));
    lm = oracle_logmf_u20(ffadd2_f2_f2_f(w, ac), &e);
  }
  float y = fmaf((float)e, L2AF, lm);
  if (a < 0x1p-12f) y = a;
  if (!(a <= FLT_MAXF)) y = isnan(x) ? NAN : INFINITY;
  return canonf(copysignf(y, x));
}
float oracle_acosh_u35_f32(float x) {
  float xc = (x >= 1.0f && x <= FLT_MAXF) ? x : 1.0f;
  int e;
  float lm;
  if (xc > 0x1p60f) {
    lm = oracle_logmf_u20(ff(xc, 0.0f), &e);
    e += 1;
  } else {
    ff_t d = ffmul_f2_f2_f2(ffadd2_f2_f_f(xc, -1.0f), ffadd2_f2_f_f(xc, 1.0f));
    lm = oracle_logmf_u20(ffadd2_f2_f2_f(ffsqrt_f2_f2(d), xc), &e);
  }
  float y = fmaf((float)e, L2AF, lm);
  if (xc == 1.0f) y = 0.0f;
  if (!(x >= 1.0f && x <= FLT_MAXF)) y = x == INFINITY ? INFINITY : NAN;
  return canonf(y);
}
float oracle_atanh_u35_f32(float x) {
  float a = fabsf(x);
  float ac = a < 1.0f ? a : 0.5f;
  ff_t q = ffdiv_f2_f2_f2(ffadd2_f2_f_f(1.0f, ac), ffadd2_f2_f_f(1.0f, -ac));
  int e;
  float lm = oracle_logmf_u20(q, &e);
  float y = 0.5f * fmaf((float)e, L2AF, lm);
  if (a < 0x1p-12f) y = a;
  if (!(a < 1.0f)) y = a == 1.0f ? INFINITY : NAN;
  return canonf(copysignf(y, x));
}

/* ---------------- pow ---------------- */
/* e^Y for an FF Y: overflow to +inf, underflow with subnormals rounded once */
static float expkf(ff_t Y) {
  if (!(fabsf(Y.x) <= 160.0f)) return Y.x > 0 ? INFINITY : 0.0f;
  float k;
  ff_t o = oracle_expf_parts(Y, &k);
  return oracle_scale2f(o.x + o.y, (int)k);
}
float oracle_pow_u10_f32(float x, float y) {
  float ax = fabsf(x);
  float axc = (ax > 0 && ax <= FLT_MAXF) ? ax : 1.0f;
  float yc = isfinite(y) ? y : 0.0f;
  int yint = isfinite(y) && y == truncf(y);
  int yodd = yint && fabsf(y) < 0x1p24f && ((int32_t)y & 1);
  float r = expkf(ffmul_f2_f2_f(oracle_logkf(ff(axc, 0.0f)), yc));
  if (x < 0 && yodd) r = -r;
  if (x < 0 && isfinite(x) && isfinite(y) && !yint) r = NAN;
  if (x == 0) {
    if (y < 0) r = yodd ? copysignf(INFINITY, x) : INFINITY;
    else if (y > 0) r = yodd ? x : 0.0f;
  }
  if (isinf(y)) {
    if (ax == 1) r = 1.0f;
    else r = ((ax < 1) == (y < 0)) ? INFINITY : 0.0f;
  }
  if (isinf(x)) {
    if (x > 0) r = y < 0 ? 0.0f : INFINITY;
    else if (y < 0) r = yodd ? -0.0f : 0.0f;
    else r = yodd ? -INFINITY : INFINITY;
  }
  if (isnan(x) || isnan(y)) r = NAN;
  if (y == 0 || x == 1) r = 1.0f;
  return canonf(r);
}
float oracle_pow_u35_f32(float x, float y) { return oracle_pow_u10_f32(x, y); }

/* ---------------- cbrt ---------------- */
static float cbrtf_core(float x, int u10) {
  float a0 = fabsf(x);
  int fin = isfinite(x) && x != 0;
  if (!fin) a0 = 1.0f;
  int off = 0;
  if (a0 < 0x1p-126f) { a0 *= 0x1p24f; off = 8; }
  int e = ilogbf(a0);
  int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  int i = e - 3 * q;
  float m = ldexpf(a0, -e);
  float a = m * ldexpf(1.0f, i);
  float c = i == 0 ? 1.0f : (i == 1 ? 0x1.965feap-1f : 0x1.428a30p-1f);
  float z = poly_f(m - 1.5f, CBRTF, 4) * c;
  float z3 = (z * z) * z;
  z = fmaf(z * fmaf(-a, z3, 1.0f), THIRDF, z);
  float zz = z * z;
  float y = a * zz;
  float d;
  if (u10) {
    ff_t y3 = ffmul_f2_f2_f(ffmul_f2_f_f(y, y), y);
    d = (y3.x - a) + y3.y;
  } else {
    d = fmaf(y * y, y, -a);
  }
  y = fmaf(-d, zz * THIRDF, y);
  y = y * ldexpf(1.0f, q - off);
  if (!fin) y = x + x;
  return canonf(copysignf(y, x));
}
float oracle_cbrt_u10_f32(float x) { return cbrtf_core(x, 1); }
float oracle_cbrt_u35_f32(float x) { return cbrtf_core(x, 0); }

/* ---------------- erfc ---------------- */
float oracle_erfc_u10_f32(float x) {
  float a = fabsf(x), y;
  if (a < 1.0f) {
    ff_t e = oracle_erfcf_a(a);
    if (x > 0) e = ff(-e.x, -e.y);
    ff_t r = ffadd2_f2_f_f2(1.0f, e);
    y = r.x + r.y;
  } else if (a <= 10.1f) {       /* F e^(-x^2) with log F = L(x) */
    ff_t E = ffadd2_f2_f2_f2(ffmul_f2_f_f(-a, a), oracle_erfcf_L(a));
    float k;
    ff_t c = oracle_expf_parts(E, &k);
    if (x > 0) {
      y = oracle_scale2f(c.x + c.y, (int)k);
    } else if (a < 4.0f) {
      c = ffscale_f2_f2_f(c, ldexpf(1.0f, (int)k));
      ff_t r = ffadd2_f2_f_f2(2.0f, ff(-c.x, -c.y));
      y = r.x + r.y;
    } else {
      y = 2.0f;
    }
  } else {
    y = x > 0 ? 0.0f : 2.0f;
  }
  if (isnan(x)) y = NAN;
  return canonf(y);
}
float oracle_erfc_u35_f32(float x) { return oracle_erfc_u10_f32(x); }
