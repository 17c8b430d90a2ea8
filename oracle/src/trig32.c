/*
 * FP32 sin and cos of the oracle in float-float (FF) arithmetic, u10 and u35.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * The paper describes the FP64 functions; these mirror Section 5.1 with
 * binary32 operations only (no FP64 anywhere):
 *   |x| < 125   Cody-Waite with pi/2 split in three floats (head by fmaf,
 *               exact; second by an exact FF product; third into the tail);
 *   |x| < 2^20  the same with a fourth constant, the third as an FF product;
 *   otherwise   the Payne-Hanek reduction of Section 5.8 in FF over the FP32
 *               table (E = 0..127, four 24-bit words, 2^64 scaling above
 *               E = 64) with the half-turn parity fix; non-finite x -> NaN.
 * sin s = s + s t (c1 + t P(t)) on the half-turn grid, the leading products
 * in FF for u10 and plain binary32 for u35.
 */
#include "common.h"
#include "coeffs32.h"

#define PIO2F_A 0x1.921fb6p0f
#define PIO2F_B (-0x1.777a5cp-25f)
#define PIO2F_C (-0x1.ee59dap-50f)
#define PIO2F_D 0x1.98a2e0p-77f
#define R_1_PIF 0x1.45f306p-2f
#define TWOPIF_H 0x1.921fb6p2f
#define TWOPIF_L (-0x1.777a5cp-23f)

extern const float *oracle_ph_tabf(void);
extern const uint8_t *oracle_ph_ibitf(void);

/* Payne-Hanek in FF: s in [-pi/4, pi/4] and the quarter-turn count mod 4
 * (the steps of the FP64 form, in float-float) */
ff_t oracle_ph_reduce_ff(float d, int *qo) {
  const float *tab = oracle_ph_tabf();
  float df = isfinite(d) ? d : 0.0f;
  int ex = ilogbf(df), M = ex > 64 ? -66 : -2;
  if (ex < 0) ex = 0;
  if (ex > 127) ex = 127;
  float u = ldexpf(df, M);
  ff_t x = ff(0, 0);
  int q = 0;
  for (int i = 0; i < 4; i++) {
    ff_t y = ffmul_f2_f_f(u, tab[ex * 4 + i]);
    x = i == 0 ? y : ffadd2_f2_f2_f2(x, y);
    float r = rintf(ldexpf(x.x, 2));
    q += low2_of_integralf(r);
    x.x = fmaf(r, -0.25f, x.x);
    x = ffnormalize_f2_f2(x);
  }
  x = ffmul_f2_f2_f2(x, ff(TWOPIF_H, TWOPIF_L));
  q += 2 * (int)(fbits(df) & oracle_ph_ibitf()[ex] & 1);
  if (!isfinite(d)) x.x = NAN;
  *qo = q & 3;
  return x;
}

/* quarter-turn Cody-Waite for |x| < 125 and for |x| < 2^20 */
static ff_t cw1f(float x, float Q) {
  float u = fmaf(Q, -PIO2F_A, x);
  ff_t h = ffmul_f2_f_f(Q, -PIO2F_B);
  ff_t s = ffadd2_f2_f_f2(u, h);
  s.y = fmaf(Q, -PIO2F_C, s.y);
  return s;
}
/* cos at |x| < 1 (Q = +-1): the fmaf head is not exact there (x is finer
 * grained than x - Q A), so Q A is an exact FF product added with TwoSum */
static ff_t cw1f_exact(float x, float Q) {
  ff_t s = ffadd2_f2_f_f2(x, ffmul_f2_f_f(Q, -PIO2F_A));
  s = ffadd2_f2_f2_f2(s, ffmul_f2_f_f(Q, -PIO2F_B));
  s.y = fmaf(Q, -PIO2F_C, s.y);
  return s;
}
static ff_t cw2f(float x, float Q) {
  float u = fmaf(Q, -PIO2F_A, x);
  ff_t s = ffadd2_f2_f_f2(u, ffmul_f2_f_f(Q, -PIO2F_B));
  s = ffadd2_f2_f2_f2(s, ffmul_f2_f_f(Q, -PIO2F_C));
  s.y = fmaf(Q, -PIO2F_D, s.y);
  return s;
}
static ff_t ph_foldf(ff_t r, int *q, int parity) {
  if ((*q & 1) != parity) {
    float sg = r.x >= 0 ? -1.0f : 1.0f;
    r = ffadd_f2_f2_f2(ff(sg * PIO2F_A, sg * PIO2F_B), r);
    *q -= (int)sg;
  }
  return r;
}
/* half-turn reduction (parity 0: sin, q even; 1: cos, q odd) */
static ff_t reduce_halff(float x, int parity, int *q) {
  float ax = fabsf(x);
  if (ax < 0x1p20f) {
    float k = parity ? rintf(fmaf(x, R_1_PIF, -0.5f)) : rintf(x * R_1_PIF);
    float Q = parity ? 2.0f * k + 1.0f : 2.0f * k;
    *q = (int)((int32_t)Q & 3);
    if (parity && ax < 1.0f) return cw1f_exact(x, Q);
    return ax < 125.0f ? cw1f(x, Q) : cw2f(x, Q);
  }
  ff_t r = oracle_ph_reduce_ff(x, q);
  return ph_foldf(r, q, parity);
}

static const float SINF_U10[4] = { SINF_U10_COEFFS };
static const float SINF_U35[5] = { SINF_U35_COEFFS };

static float sinf_poly_u10(ff_t s) {
  ff_t t = ffsqu_f2_f2(s);
  float p = poly_f(t.x, SINF_U10, 4);
  ff_t w = ffadd_f2_f2_f(ff(SINF_U10_C1H, SINF_U10_C1L), t.x * p);
  w = ffmul_f2_f2_f2(t, w);
  w = ffmul_f2_f2_f2(s, w);
  ff_t r = ffadd_f2_f2_f2(s, w);
  return r.x + r.y;
}
static float sinf_poly_u35(float s) {
  float t = s * s;
  return fmaf(s * t, poly_f(t, SINF_U35, 5), s);
}

float oracle_sin_u10_f32(float x) {
  int q;
  ff_t s = reduce_halff(x, 0, &q);
  float y = sinf_poly_u10(s);
  if (q & 2) y = -y;
  if (x == 0) y = x;
  return canonf(y);
}
float oracle_cos_u10_f32(float x) {
  int q;
  ff_t s = reduce_halff(x, 1, &q);
  float y = sinf_poly_u10(s);
  if (!(q & 2)) y = -y;
  return canonf(y);
}
float oracle_sin_u35_f32(float x) {
  int q;
  ff_t s = reduce_halff(x, 0, &q);
  float y = sinf_poly_u35(s.x + s.y);
  if (q & 2) y = -y;
  if (x == 0) y = x;
  return canonf(y);
}
float oracle_cos_u35_f32(float x) {
  int q;
  ff_t s = reduce_halff(x, 1, &q);
  float y = sinf_poly_u35(s.x + s.y);
  if (!(q & 2)) y = -y;
  return canonf(y);
}

/* exported for the brute-force reduction pin */
void oracle_ph_reduce_f32(float x, int *q, float *hi, float *lo) {
  ff_t r = oracle_ph_reduce_ff(x, q);
  *hi = r.x;
  *lo = r.y;
}

/* ---------------- tan, sincos (quarter-turn reduction) ----------------
 * s = x - Q pi/2 in [-pi/4, pi/4] with Q = rint(x 2/pi) (Cody-Waite levels
 * as above; Payne-Hanek's quarter turns beyond 2^20).  tan s = s + s t (c1 +
 * t P(t)) with the leading products in FF (u10), -1/tan s for odd Q;
 * sincos from one reduction: sin s as above and cos s = 1 - t/2 + t^2 C(t)
 * (FF for u10), swapped and signed by Q mod 4. */
#define R_2_PIF 0x1.45f306p-1f
static const float TANF_P10[8] = { TANF_U10_COEFFS };
static const float TANF_P35[8] = { TANF_U35_COEFFS };
static const float COSF_P[3] = { COSF_U10_COEFFS };

static ff_t reduce_quarterf(float x, int *q) {
  float ax = fabsf(x);
  if (ax < 0x1p20f) {
    float Q = rintf(x * R_2_PIF);
    *q = (int)((int32_t)Q & 3);
    return ax < 125.0f ? cw1f(x, Q) : cw2f(x, Q);
  }
  ff_t r = oracle_ph_reduce_ff(x, q);
  *q &= 3;
  return r;
}

float oracle_tan_u10_f32(float x) {
  int q;
  ff_t s = reduce_quarterf(x, &q);
  ff_t t = ffsqu_f2_f2(s);
  float p = poly_f(t.x, TANF_P10, 8);
  ff_t w = ffadd_f2_f2_f(ff(TANF_U10_C1H, TANF_U10_C1L), t.x * p);
  w = ffmul_f2_f2_f2(s, ffmul_f2_f2_f2(t, w));
  ff_t r = ffadd_f2_f2_f2(s, w);
  if (q & 1) r = ffdiv_f2_f2_f2(ff(-1.0f, 0.0f), r);
  float y = r.x + r.y;
  if (x == 0) y = x;
  return canonf(y);
}
float oracle_tan_u35_f32(float x) {
  int q;
  ff_t s = reduce_quarterf(x, &q);
  float s1 = s.x + s.y, t = s1 * s1;
  float r = fmaf(s1 * t, poly_f(t, TANF_P35, 8), s1);
  if (q & 1) r = -1.0f / r;
  if (x == 0) r = x;
  return canonf(r);
}

static void sincos_out(int q, float sn, float cs, float x, float *os, float *oc) {
  float a = (q & 1) ? cs : sn, b = (q & 1) ? sn : cs;
  if (q == 1 || q == 2) b = -b;
  if (q & 2) a = -a;
  if (x == 0) a = x;
  *os = canonf(a);
  *oc = canonf(b);
}
void oracle_sincos_u10_f32(float x, float *os, float *oc) {
  int q;
  ff_t s = reduce_quarterf(x, &q);
  float sn = sinf_poly_u10(s);
  ff_t t = ffsqu_f2_f2(s);
  float v = (t.x * t.x) * poly_f(t.x, COSF_P, 3);
  ff_t c = ffadd2_f2_f_f2(1.0f, ffscale_f2_f2_f(t, -0.5f));
  c = ffadd_f2_f2_f(c, v);
  sincos_out(q, sn, c.x + c.y, x, os, oc);
}
void oracle_sincos_u35_f32(float x, float *os, float *oc) {
  int q;
  ff_t s = reduce_quarterf(x, &q);
  float s1 = s.x + s.y, t = s1 * s1;
  float sn = sinf_poly_u35(s1);
  float cs = fmaf(t * t, poly_f(t, COSF_P, 3), fmaf(t, -0.5f, 1.0f));
  sincos_out(q, sn, cs, x, os, oc);
}
