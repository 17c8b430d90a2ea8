/*
 * FP32 tgamma and lgamma of the oracle (u10; u35 runs the same algorithm):
 * the FP64 design of gamma64.c in float-float arithmetic with binary32
 * coefficients: Stirling from 8 with the FF logarithm of powf, polynomials
 * about 2 and 1.5, the shift y -> y + n, the reflection with sin(pi x)
 * reduced exactly, tgamma = exp of the FF log-gamma.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#include "common.h"
#include "coeffs32.h"
#include "explog32.h"

#define LOG2PI_HF 0x1.d67f1cp-1f
#define LOG2PI_LF 0x1.0c97d6p-26f
#define LOGPI_HF 0x1.250d04p+0f
#define LOGPI_LF 0x1.1cf438p-25f
#define PI_HF 0x1.921fb6p+1f
#define PI_LF (-0x1.777a5cp-24f)
/* 64 ln 2 as an FF: 64 times the 15-bit head of ln 2 and 64 times its tail (both exact) */
#define LN2X64_HF 0x1.62e4p+5f
#define LN2X64_LF 0x1.7f7d1cp-14f

static const float LGR_H[4] = { LGF_R2_HEAD };
static const float LGR_P[8] = { LGF_R2_COEFFS };
static const float LGM_H[6] = { LGF_M_HEAD };
static const float LGM_P[7] = { LGF_M_COEFFS };
static const float LGS_P[4] = { LGF_ST_COEFFS };
static const float SPI_H[4] = { SINPIF_HEAD };
static const float SPI_P[5] = { SINPIF_COEFFS };

static ff_t fneg(ff_t a) { return ff(-a.x, -a.y); }

static ff_t lgf_r2(ff_t e) {
  float p = poly_f(e.x, LGR_P, 8);
  ff_t in = ffadd2_f2_f2_f(ff(LGR_H[2], LGR_H[3]), e.x * p);
  in = ffadd2_f2_f2_f2(ff(LGR_H[0], LGR_H[1]), ffmul_f2_f2_f2(in, e));
  return ffmul_f2_f2_f2(in, e);
}
static ff_t lgf_m(ff_t u) {
  float p = poly_f(u.x, LGM_P, 7);
  ff_t in = ffadd2_f2_f2_f(ff(LGM_H[4], LGM_H[5]), u.x * p);
  in = ffadd2_f2_f2_f2(ff(LGM_H[2], LGM_H[3]), ffmul_f2_f2_f2(in, u));
  return ffadd2_f2_f2_f2(ff(LGM_H[0], LGM_H[1]), ffmul_f2_f2_f2(in, u));
}
static ff_t lgf_stirling(ff_t y) {
  ff_t ly = oracle_logkf(y);
  ff_t r = ffmul_f2_f2_f2(ffadd2_f2_f2_f(y, -0.5f), ly);
  r = ffadd2_f2_f2_f2(r, fneg(y));
  r = ffadd2_f2_f2_f2(r, ff(LOG2PI_HF, LOG2PI_LF));
  float w = 1.0f / (y.x * y.x);
  return ffadd2_f2_f2_f(r, poly_f(w, LGS_P, 4) / y.x);
}
static ff_t lgammaf_pos(ff_t y) {
  if (y.x >= 8) return lgf_stirling(y);
  if (y.x >= 1.75f && y.x < 2.5f) return lgf_r2(ffnormalize_f2_f2(ffadd2_f2_f2_f(y, -2.0f)));
  if (y.x >= 1.25f && y.x < 1.75f) return lgf_m(ffnormalize_f2_f2(ffadd2_f2_f2_f(y, -1.5f)));
  if (y.x >= 0.5f && y.x < 1.25f) {
    ff_t r = y.x < 0.75f ? lgf_m(ffnormalize_f2_f2(ffadd2_f2_f2_f(y, -0.5f)))
                         : lgf_r2(ffnormalize_f2_f2(ffadd2_f2_f2_f(y, -1.0f)));
    return ffadd2_f2_f2_f2(r, fneg(oracle_logkf(y)));
  }
  int n = (int)(8.0f - floorf(y.x));
  ff_t P = y, z = y;
  for (int i = 1; i < n; i++) {
    z = ffadd2_f2_f2_f(z, 1.0f);
    P = ffmul_f2_f2_f2(P, z);
  }
  ff_t s = lgf_stirling(ffadd2_f2_f2_f(y, (float)n));
  return ffadd2_f2_f2_f2(s, fneg(oracle_logkf(P)));
}
static ff_t sinpif_ff(float x) {
  float r = x - 2.0f * rintf(0.5f * x);
  float s = r > 0.5f ? 1.0f - r : (r < -0.5f ? -1.0f - r : r);
  ff_t T = ffmul_f2_f_f(s, s);
  float p = poly_f(T.x, SPI_P, 5);
  ff_t in = ffadd2_f2_f2_f(ff(SPI_H[2], SPI_H[3]), T.x * p);
  in = ffadd2_f2_f2_f2(ff(SPI_H[0], SPI_H[1]), ffmul_f2_f2_f2(T, in));
  return ffmul_f2_f2_f(in, s);
}
static ff_t lgammaf_ff(float x, int *sign) {
  *sign = 1;
  if (x > 0) return lgammaf_pos(ff(x, 0.0f));
  /* |x| < 2^-100: sin(pi x) is pi x to far below an ulp and pi x would lose
   * its precision in the subnormal range; formed from x 2^64 (exact), with
   * 64 ln 2 taken off its logarithm */
  int up = fabsf(x) < 0x1p-100f;
  ff_t sp = up ? ffmul_f2_f2_f(ff(PI_HF, PI_LF), ldexpf(x, 64)) : sinpif_ff(x);
  *sign = sp.x < 0 ? -1 : 1;
  ff_t l = oracle_logkf(ff(fabsf(sp.x), sp.x < 0 ? -sp.y : sp.y));
  if (up) l = ffadd2_f2_f2_f2(l, ff(-LN2X64_HF, -LN2X64_LF));
  ff_t r = ffadd2_f2_f2_f2(ff(LOGPI_HF, LOGPI_LF), fneg(l));
  return ffadd2_f2_f2_f2(r, fneg(lgammaf_pos(ffadd2_f2_f_f(1.0f, -x))));
}

float oracle_lgamma_u10_f32(float x) {
  float a = fabsf(x);
  int sign;
  if (isnan(x)) return canonf(NAN);
  if (isinf(x) || x == 0 || (x < 0 && (a >= 0x1p23f || x == rintf(x)))) return INFINITY;
  if (x > 0x1p124f) return INFINITY;
  ff_t L = lgammaf_ff(x, &sign);
  float y = L.x + L.y;
  if (!isfinite(y)) y = INFINITY;
  return canonf(y);
}
float oracle_tgamma_u10_f32(float x) {
  float a = fabsf(x);
  int sign;
  if (isnan(x) || x == -INFINITY || (x < 0 && (a >= 0x1p23f || x == rintf(x)))) return canonf(NAN);
  if (x == 0) return copysignf(INFINITY, x);
  if (x > 36.0f) return INFINITY;
  if (x < -42.0f) return sinpif_ff(x).x < 0 ? -0.0f : 0.0f;
  ff_t L = lgammaf_ff(x, &sign);
  float k;
  ff_t o = oracle_expf_parts(L, &k);
  float y = oracle_scale2f(o.x + o.y, (int)k);
  return canonf(sign < 0 ? -y : y);
}
float oracle_lgamma_u35_f32(float x) { return oracle_lgamma_u10_f32(x); }
float oracle_tgamma_u35_f32(float x) { return oracle_tgamma_u10_f32(x); }
