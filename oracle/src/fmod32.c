/*
 * FP32 fmod and remainder of the oracle (exact results; u35 = u10): the
 * FP64 algorithm of fmod64.c (Section 5.9 long division, one division, the
 * partial remainder exact as a float-float pair) in binary32, with the
 * divisor scaled by 2^j while the quotient exceeds 2^100 (every pair of
 * floats, quotients up to 2^277, at most 24 steps) and subnormal divisors
 * rescaled by 2^24.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#include "common.h"

#define FMODF_MAXIT 24

static float rdownf(float v) { return nextafterf(v, 0.0f); }

static ff_t fmodf_step(ff_t r, float D, float rD) {
  float q = truncf(rdownf(r.x) * rD);
  q = (3 * D > r.x && r.x > D) ? 2 : q;
  q = (2 * D > r.x && r.x > D) ? 1 : q;
  q = r.x == D ? (r.y >= 0 ? 1 : 0) : q;
  return ffnormalize_f2_f2(ffadd2_f2_f2_f2(r, ffmul_f2_f_f(q, -D)));
}

static float fmodf_abs(float n, float d) {
  int sub = d < 0x1p-126f;
  int kmin = sub ? 24 : 0;
  float dmin = ldexpf(d, kmin);
  float rd0 = rdownf(1.0f / dmin);
  int ed = ilogbf(d);
  ff_t r = ff(n, 0);
  for (int it = 0; it < FMODF_MAXIT && r.x >= dmin; it++) {
    int j = ilogbf(r.x) - ed - 100;
    if (j < kmin) j = kmin;
    r = fmodf_step(r, ldexpf(d, j), ldexpf(rd0, kmin - j));
  }
  float ret;
  if (sub) {
    r = ff(r.x * 0x1p24f, r.y * 0x1p24f);
    for (int k = 0; k < 4 && r.x >= dmin; k++) r = fmodf_step(r, dmin, rd0);
    ret = r.x * 0x1p-24f;
    if (r.x + r.y == dmin) ret = 0;
  } else {
    ret = r.x;
    if (r.x + r.y == d) ret = 0;
  }
  return ret;
}

float oracle_fmod_u10_f32(float x, float y) {
  float n = fabsf(x), d = fabsf(y);
  int ok = isfinite(n) && d > 0 && isfinite(d);
  float ret = fmodf_abs(ok ? n : 0.0f, ok ? d : 1.0f);
  ret = copysignf(ret, x);
  if (n < d) ret = x;
  if (!(d > 0) || isinf(n) || isnan(x) || isnan(y)) ret = NAN;
  return canonf(ret);
}
float oracle_fmod_u35_f32(float x, float y) { return oracle_fmod_u10_f32(x, y); }

float oracle_remainder_u10_f32(float x, float y) {
  float n = fabsf(x), d = fabsf(y);
  int ok = isfinite(n) && d > 0 && isfinite(d);
  float nn = ok ? n : 0.0f, dd2 = ok ? d : 1.0f;
  float r2 = nn;
  if (dd2 <= 0x1.fffffep126f) r2 = fmodf_abs(nn, 2 * dd2);
  if (r2 + r2 > dd2) {
    r2 = r2 - dd2;
    if (r2 + r2 >= dd2) r2 = r2 - dd2;
  }
  float ret = signbit(x) ? -r2 : r2;
  if (isinf(y) && isfinite(x)) ret = x;
  if (!(d > 0) || isinf(n) || isnan(x) || isnan(y)) ret = NAN;
  return canonf(ret);
}
float oracle_remainder_u35_f32(float x, float y) { return oracle_remainder_u10_f32(x, y); }
