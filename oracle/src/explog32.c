/*
 * FP32 exp, log, log1p, tanh and erf of the oracle (float-float where the
 * 1-ULP bound needs it), u10 and u35.  binary32 operations only.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * exp    Section 5.6 in binary32: x = k ln2 + r, polynomial, 2^k in two steps;
 *        u10 keeps the residual of r and forms 1 + r in FF.
 * log    Section 5.5 in binary32: m in [0.75, 1.5), z = 2(m-1)/(m+1) in FF.
 * log1p  1 + x as an FF pair, then the log reduction applied to the pair.
 * tanh   expm1(2|x|) / (expm1(2|x|) + 2) in FF, expm1 from the exp reduction.
 * erf    |x| < 1: x (c0 + t (c1 + t P(t))), t = x^2, with c0, t and the
 *        two leading terms in FF;
 *        1 <= |x| < 3.95: 1 - exp(-x^2 + L(|x|)), L = log(erfc(x) e^(x^2))
 *        a polynomial in u = |x| - 2.475 with its constant term in FF, -x^2
 *        exact in FF, the exponential of the FF sum; |x| >= 3.95 rounds to +-1.
 */
#include "common.h"
#include "coeffs32.h"

#define R_LN2F 0x1.715476p0f
#define L2AF 0x1.62e430p-1f
#define L2BF (-0x1.05c610p-29f)
#define L2HF 0x1.62e400p-1f       /* ln2 to 15 bits: e*L2HF exact for |e| < 2^9 */
#define L2LF 0x1.7f7d1cp-20f

static float pow2if(int k) { return ldexpf(1.0f, k); }
static float scale2f(float y, int k) {   /* as scale2 of the FP64 file */
  int k1 = k / 2, k2 = k - k1;
  return ldexpf(ldexpf(y, k1), k2);
}

/* ---------------- exp ---------------- */
static const float EXPF_U10[6] = { EXPF_U10_COEFFS };
static const float EXPF_U35[5] = { EXPF_U35_COEFFS };

static float expf_sel(float x, float y) {
  if (!(fabsf(x) <= 104.0f)) y = x > 0 ? INFINITY : (x < 0 ? 0.0f : NAN);
  return canonf(y);
}
float oracle_exp_u10_f32(float x) {
  float xc = fabsf(x) <= 104.0f ? x : 0.0f;
  float k = rintf(xc * R_LN2F);
  float h = fmaf(k, -L2AF, xc);
  float r = fmaf(k, -L2BF, h);
  float rl = fmaf(k, -L2BF, h - r);
  float w = fmaf(r * r, poly_f(r, EXPF_U10, 6), rl);
  ff_t o = ffadd_f2_f_f(1.0f, r);
  return expf_sel(x, scale2f(o.x + (o.y + w), (int)k));
}
float oracle_exp_u35_f32(float x) {
  float xc = fabsf(x) <= 104.0f ? x : 0.0f;
  float k = rintf(xc * R_LN2F);
  float r = fmaf(k, -L2BF, fmaf(k, -L2AF, xc));
  float v = fmaf(r * r, poly_f(r, EXPF_U35, 5), r);
  return expf_sel(x, scale2f(1.0f + v, (int)k));
}

/* e^(h + l) as an FF pair for an FF argument with |h| <= 104 and a normal
 * result (the exponential of erf's tail) */
static ff_t expf_ff(ff_t a) {
  float k = rintf(a.x * R_LN2F);
  float h = fmaf(k, -L2AF, a.x);
  ff_t r = ffadd2_f2_f_f(h, fmaf(k, -L2BF, a.y));
  float w = fmaf(r.x * r.x, poly_f(r.x, EXPF_U10, 6), r.y);
  ff_t o = ffadd_f2_f_f(1.0f, r.x);
  return ffscale_f2_f2_f(ff(o.x, o.y + w), pow2if((int)k));
}

/* ---------------- log, log1p ---------------- */
static const float LOGF_U10[4] = { LOGF_U10_COEFFS };
static const float LOGF_U35[3] = { LOGF_U35_COEFFS };

/* a > 0 finite: a = m 2^e, m in [0.75, 1.5) (subnormals scaled by 2^32) */
static float logf_reduce(float a, int *e) {
  int off = 0;
  if (a < 0x1p-126f) { a *= 0x1p32f; off = 32; }
  int ex = ilogbf(a);
  float m = ldexpf(a, -ex);
  if (m >= 1.5f) { m *= 0.5f; ex++; }
  *e = ex - off;
  return m;
}
static float logf_special(float x, float y) {
  if (x == 0) return -INFINITY;
  if (x < 0 || isnan(x)) return NAN;
  if (isinf(x)) return INFINITY;
  return y;
}
/* e ln2 + log(m + ml) in FF; z = 2 (m + ml - 1) / (m + ml + 1) */
static ff_t logf_core_u10(float m, float ml, int e) {
  ff_t num = ffscale_f2_f2_f(ffadd2_f2_f_f(m - 1.0f, ml), 2.0f);
  ff_t den = ffadd2_f2_f_f2(1.0f, ff(m, ml));
  ff_t z = ffdiv_f2_f2_f2(num, den);
  float t = z.x * z.x;
  float corr = (z.x * t) * poly_f(t, LOGF_U10, 4);
  float ed = (float)e;
  ff_t r = ffadd_f2_f2_f2(ff(ed * L2HF, ed * L2LF), z);
  return ffadd_f2_f2_f(r, corr);
}
float oracle_log_u10_f32(float x) {
  float a = (x > 0 && x <= 0x1.fffffep127f) ? x : 1.0f;
  int e;
  float m = logf_reduce(a, &e);
  ff_t r = logf_core_u10(m, 0.0f, e);
  return canonf(logf_special(x, r.x + r.y));
}
float oracle_log_u35_f32(float x) {
  float a = (x > 0 && x <= 0x1.fffffep127f) ? x : 1.0f;
  int e;
  float m = logf_reduce(a, &e);
  float z = (2.0f * (m - 1.0f)) / (1.0f + m);
  float t = z * z;
  float lm = fmaf(z * t, poly_f(t, LOGF_U35, 3), z);
  return canonf(logf_special(x, fmaf((float)e, L2AF, lm)));
}

static float log1pf_special(float x, float y) {
  if (x == -1.0f) return -INFINITY;
  if (x < -1.0f || isnan(x)) return NAN;
  if (isinf(x)) return INFINITY;
  if (x == 0) return x;
  return y;
}
float oracle_log1p_u10_f32(float x) {
  float xc = (x > -1.0f && x <= 0x1.fffffep127f) ? x : 0.0f;
  ff_t s = ffadd2_f2_f_f(1.0f, xc);
  int e;
  float m = logf_reduce(s.x, &e);
  float ml = ldexpf(s.y, -e);
  ff_t r = logf_core_u10(m, ml, e);
  return canonf(log1pf_special(x, r.x + r.y));
}
float oracle_log1p_u35_f32(float x) {
  float xc = (x > -1.0f && x <= 0x1.fffffep127f) ? x : 0.0f;
  ff_t s = ffadd2_f2_f_f(1.0f, xc);
  int e;
  float m = logf_reduce(s.x, &e);
  float ml = ldexpf(s.y, -e);
  float z = (2.0f * ((m - 1.0f) + ml)) / ((1.0f + m) + ml);
  float t = z * z;
  float lm = fmaf(z * t, poly_f(t, LOGF_U35, 3), z);
  return canonf(log1pf_special(x, fmaf((float)e, L2AF, lm)));
}

/* ---------------- tanh ---------------- */
static const float EXPM1F[5] = { EXPM1F_COEFFS };

/* expm1(a) in FF for 0 <= a <= 18.2: 2^k (e^r - 1) + (2^k - 1) */
static ff_t expm1f_ff(float a) {
  float k = rintf(a * R_LN2F);
  float h = fmaf(k, -L2AF, a);
  float r = fmaf(k, -L2BF, h);
  float rl = fmaf(k, -L2BF, h - r);
  ff_t rr = ff(r, rl);
  ff_t q = ffscale_f2_f2_f(ffsqu_f2_f2(rr), 0.5f);
  float v = ((r * r) * r) * poly_f(r, EXPM1F, 5);
  ff_t s = ffadd2_f2_f2_f2(rr, q);
  s = ffadd2_f2_f2_f(s, v);
  float p = pow2if((int)k);
  ff_t t = ffadd2_f2_f2_f(ffscale_f2_f2_f(s, p), p);       /* 2^k e^r */
  return ffnormalize_f2_f2(ffadd2_f2_f2_f(t, -1.0f));      /* - 1 */
}
float oracle_tanh_u10_f32(float x) {
  float a = fabsf(x);
  float ac = a < 9.1f ? a : 0.0f;
  ff_t em = expm1f_ff(2.0f * ac);
  ff_t r = ffdiv_f2_f2_f2(em, ffadd2_f2_f2_f(em, 2.0f));
  float y = r.x + r.y;
  if (!(a < 9.1f)) y = 1.0f;
  y = copysignf(y, x);
  if (isnan(x)) y = NAN;
  return canonf(y);
}
float oracle_tanh_u35_f32(float x) {
  float a = fabsf(x);
  float ac = a < 9.1f ? a : 0.0f;
  ff_t em = expm1f_ff(2.0f * ac);
  float e = em.x + em.y;
  float y = e / (e + 2.0f);
  if (!(a < 9.1f)) y = 1.0f;
  y = copysignf(y, x);
  if (isnan(x)) y = NAN;
  return canonf(y);
}

/* ---------------- erf ---------------- */
static const float ERFF_A[7] = { ERFF_A_COEFFS };
static const float ERFF_B[11] = { ERFF_B_COEFFS };
#define ERF_C 2.475f

float oracle_erf_u10_f32(float x) {
  float a = fabsf(x), y;
  if (a < 1.0f) {
    ff_t t = ffmul_f2_f_f(a, a);
    float p = poly_f(t.x, ERFF_A + 1, 6);                       /* c2 + c3 t + ... */
    ff_t w1 = ffadd_f2_f_f(ERFF_A[0], t.x * p);                  /* c1 + t P2(t) */
    ff_t w = ffadd_f2_f2_f2(ff(ERFF_A_C1H, ERFF_A_C1L), ffmul_f2_f2_f2(t, w1));
    ff_t r = ffmul_f2_f2_f(w, a);
    y = r.x + r.y;
    if (a < 0x1p-30f) {            /* x 2/sqrt(pi) at a scale where a * c0lo is not lost */
      float as = a * 0x1p32f;
      y = fmaf(as, ERFF_A_C1H, as * ERFF_A_C1L) * 0x1p-32f;
    }
  } else {
    float ac = a < 3.95f ? a : 1.0f;
    float u = ac - ERF_C;
    ff_t e = ffadd2_f2_f2_f2(ffmul_f2_f_f(-ac, ac), ff(ERFF_B_C1H, ERFF_B_C1L));
    e = ffadd2_f2_f2_f(e, u * poly_f(u, ERFF_B, 11));
    ff_t c = expf_ff(e);
    ff_t d = ffadd2_f2_f_f2(1.0f, ff(-c.x, -c.y));
    y = d.x + d.y;
    if (!(a < 3.95f)) y = 1.0f;
  }
  y = copysignf(y, x);
  if (isnan(x)) y = NAN;
  return canonf(y);
}
float oracle_erf_u35_f32(float x) {
  float a = fabsf(x), y;
  if (a < 1.0f) {
    float t = a * a;
    float p = fmaf(t, poly_f(t, ERFF_A, 7), ERFF_A_C1H);
    y = p * a;
  } else {
    float ac = a < 3.95f ? a : 1.0f;
    float u = ac - ERF_C;
    ff_t e = ffadd2_f2_f2_f2(ffmul_f2_f_f(-ac, ac), ff(ERFF_B_C1H, ERFF_B_C1L));
    e = ffadd2_f2_f2_f(e, u * poly_f(u, ERFF_B, 11));
    ff_t c = expf_ff(e);
    y = 1.0f - (c.x + c.y);
    if (!(a < 3.95f)) y = 1.0f;
  }
  y = copysignf(y, x);
  if (isnan(x)) y = NAN;
  return canonf(y);
}

/* ---------------- cores shared with the other FP32 functions ---------------- */
static const float POWLOGF[5] = { POWLOGF_COEFFS };

float oracle_scale2f(float y, int k) { return scale2f(y, k); }

/* 2^k (1 + r + rl) with the 1-ULP polynomial, |r| <= ln2/2 */
float oracle_expf_tail_u10(float r, float rl, float k) {
  float w = fmaf(r * r, poly_f(r, EXPF_U10, 6), rl);
  ff_t o = ffadd_f2_f_f(1.0f, r);
  return scale2f(o.x + (o.y + w), (int)k);
}

/* e^(a.x + a.y) = o 2^k with o an FF pair in [0.7, 1.42], for |a.x| <= 160 */
ff_t oracle_expf_parts(ff_t a, float *kp) {
  float k = rintf(a.x * R_LN2F);
  float h = fmaf(k, -L2AF, a.x);
  ff_t r = ffadd2_f2_f_f(h, fmaf(k, -L2BF, a.y));
  float w = fmaf(r.x * r.x, poly_f(r.x, EXPF_U10, 6), r.y);
  ff_t o = ffadd_f2_f_f(1.0f, r.x);
  *kp = k;
  return ff(o.x, o.y + w);
}

/* e^r - 1 as an FF pair and k with a = k ln2 + r, |a| <= 160 */
ff_t oracle_expm1f_s(float a, float *kp) {
  float k = rintf(a * R_LN2F);
  float h = fmaf(k, -L2AF, a);
  float r = fmaf(k, -L2BF, h);
  float rl = fmaf(k, -L2BF, h - r);
  ff_t rr = ff(r, rl);
  ff_t q = ffscale_f2_f2_f(ffsqu_f2_f2(rr), 0.5f);
  float v = ((r * r) * r) * poly_f(r, EXPM1F, 5);
  ff_t s = ffadd2_f2_f2_f2(rr, q);
  *kp = k;
  return ffadd2_f2_f2_f(s, v);
}

/* FF argument a > 0 (finite): log m as an FF pair with a = m 2^e, m in
 * [0.75, 1.5) (the u10 core without e ln2) */
ff_t oracle_logmf_u10(ff_t a, int *ep) {
  int e;
  float m = logf_reduce(a.x, &e);
  float ml = ldexpf(a.y, -e);
  ff_t num = ffscale_f2_f2_f(ffadd2_f2_f_f(m - 1.0f, ml), 2.0f);
  ff_t den = ffadd2_f2_f_f2(1.0f, ff(m, ml));
  ff_t z = ffdiv_f2_f2_f2(num, den);
  float t = z.x * z.x;
  float corr = (z.x * t) * poly_f(t, LOGF_U10, 4);
  *ep = e;
  return ffadd_f2_f2_f(z, corr);
}

/* log m in binary32 with z = 2(m-1)/(m+1) corrected once: the residual
 * num - z (1 + m) (the rounding of 1 + m and the FF tail included) goes back
 * through the reciprocal, then the 3.5-ULP polynomial (the 3.5-ULP forms of
 * asinh, acosh, atanh) */
float oracle_logmf_u20(ff_t a, int *ep) {
  int e;
  float m = logf_reduce(a.x, &e);
  float ml = ldexpf(a.y, -e);
  float num = 2.0f * ((m - 1.0f) + ml);
  float den = 1.0f + m;
  float rd = 1.0f / den;
  float z = num * rd;
  float r = fmaf(-z, den, num) - z * (((1.0f - den) + m) + ml);
  z = fmaf(r, rd, z);
  float t = z * z;
  *ep = e;
  return fmaf(z * t, poly_f(t, LOGF_U35, 3), z);
}

/* log of an FF a > 0 as an FF pair: e ln2 + log m with the FF core */
ff_t oracle_logf_ff(ff_t a) {
  int e;
  ff_t lm = oracle_logmf_u10(a, &e);
  float ed = (float)e;
  return ffadd2_f2_f2_f2(ff(ed * L2HF, ed * L2LF), lm);
}

/* log of an FF a > 0 to about 2^-40: the internal log of powf (first
 * coefficient FF, the correction in FF products) */
ff_t oracle_logkf(ff_t a) {
  int e;
  float m = logf_reduce(a.x, &e);
  float ml = ldexpf(a.y, -e);
  ff_t num = ffscale_f2_f2_f(ffadd2_f2_f_f(m - 1.0f, ml), 2.0f);
  ff_t z = ffdiv_f2_f2_f2(num, ffadd2_f2_f_f2(1.0f, ff(m, ml)));
  ff_t t = ffsqu_f2_f2(z);
  float q = poly_f(t.x, POWLOGF, 5);
  ff_t w = ffadd_f2_f2_f(ff(POWLOGF_C1H, POWLOGF_C1L), t.x * q);
  w = ffmul_f2_f2_f2(t, w);
  w = ffmul_f2_f2_f2(z, w);
  ff_t lm = ffadd_f2_f2_f2(z, w);
  float ed = (float)e;
  return ffadd2_f2_f2_f2(ff(ed * L2HF, ed * L2LF), lm);
}

/* L(x) = log(erfc(x) e^(x^2)) as an FF pair, 1 <= x <= 10.1: c0 + u (c1 +
 * u P(u)) about 2.5 (x < 3.95) or 7, c0 and c1 FF pairs */
static const float ERFCF_B[14] = { ERFCF_B_COEFFS };
static const float ERFCF_BH[4] = { ERFCF_B_HEAD };
static const float ERFCF_C[11] = { ERFCF_C_COEFFS };
static const float ERFCF_CH[4] = { ERFCF_C_HEAD };
ff_t oracle_erfcf_L(float x) {
  int tail = x >= 3.95f;
  const float *h = tail ? ERFCF_CH : ERFCF_BH;
  float u = x - (tail ? 7.0f : 2.5f);
  float p = tail ? poly_f(u, ERFCF_C, 11) : poly_f(u, ERFCF_B, 14);
  ff_t in = ffadd2_f2_f2_f(ff(h[2], h[3]), u * p);
  return ffadd2_f2_f2_f2(ff(h[0], h[1]), ffmul_f2_f2_f(in, u));
}

/* erf(a) for 0 <= a < 1 as an FF pair with three FF levels, C0 + T (C1 + T
 * (C2 + t P(t))), T = a^2 exact (erfc's 1 - erf near 1) */
static const float ERFCF_AH[6] = { ERFCF_A_HEAD };
static const float ERFCF_A[6] = { ERFCF_A_COEFFS };
ff_t oracle_erfcf_a(float a) {
  ff_t T = ffmul_f2_f_f(a, a);
  float p = poly_f(T.x, ERFCF_A, 6);
  ff_t in = ffadd2_f2_f2_f(ff(ERFCF_AH[4], ERFCF_AH[5]), T.x * p);
  in = ffadd2_f2_f2_f2(ff(ERFCF_AH[2], ERFCF_AH[3]), ffmul_f2_f2_f2(T, in));
  in = ffadd2_f2_f2_f2(ff(ERFCF_AH[0], ERFCF_AH[1]), ffmul_f2_f2_f2(T, in));
  return ffmul_f2_f2_f(in, a);
}

/* erf(a) for 0 <= a < 1 as an FF pair (the u10 kernel) */
ff_t oracle_erff_a(float a) {
  ff_t t = ffmul_f2_f_f(a, a);
  float p = poly_f(t.x, ERFF_A + 1, 6);
  ff_t w1 = ffadd_f2_f_f(ERFF_A[0], t.x * p);
  ff_t w = ffadd_f2_f2_f2(ff(ERFF_A_C1H, ERFF_A_C1L), ffmul_f2_f2_f2(t, w1));
  return ffmul_f2_f2_f(w, a);
}
