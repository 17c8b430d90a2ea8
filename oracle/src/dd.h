/*
 * Double-double (DD) and float-float (FF) operators of the oracle.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * Semantics follow Table 5 of the paper ("DD Functions") and Section 5's
 * remark that DD values are kept un-normalized unless a step renormalizes
 * them explicitly.  Each operator below is written once, as a fixed sequence
 * of IEEE round-to-nearest operations; the formula is given beside it.
 * Compiled with -ffp-contract=off so that no multiply and add is fused
 * unless fma() is written.
 */
#ifndef ORACLE_DD_H
#define ORACLE_DD_H
#include <math.h>

typedef struct { double x, y; } dd_t;   /* value = x + y, |y| small */
typedef struct { float x, y; } ff_t;

static inline dd_t dd(double h, double l) { dd_t r; r.x = h; r.y = l; return r; }

/* x + y, |x| >= |y| (Dekker's FastTwoSum) */
static inline dd_t ddadd_d2_d_d(double x, double y) {
  double s = x + y;
  return dd(s, (x - s) + y);
}
/* x + y, any magnitudes (Knuth's TwoSum) */
static inline dd_t ddadd2_d2_d_d(double x, double y) {
  double s = x + y, v = s - x;
  return dd(s, (x - (s - v)) + (y - v));
}
/* DD + DD, |x| >= |y|:  s = x.x + y.x, lo = (x.x - s) + y.x + x.y + y.y */
static inline dd_t ddadd_d2_d2_d2(dd_t x, dd_t y) {
  double s = x.x + y.x;
  return dd(s, (((x.x - s) + y.x) + x.y) + y.y);
}
/* DD + DD, any magnitudes: TwoSum of the heads plus both tails */
static inline dd_t ddadd2_d2_d2_d2(dd_t x, dd_t y) {
  double s = x.x + y.x, v = s - x.x;
  double e = (x.x - (s - v)) + (y.x - v);
  return dd(s, (e + x.y) + y.y);
}
/* double + DD, |x| >= |y| */
static inline dd_t ddadd_d2_d_d2(double x, dd_t y) {
  double s = x + y.x;
  return dd(s, ((x - s) + y.x) + y.y);
}
/* double + DD, any magnitudes */
static inline dd_t ddadd2_d2_d_d2(double x, dd_t y) {
  double s = x + y.x, v = s - x;
  return dd(s, ((x - (s - v)) + (y.x - v)) + y.y);
}
/* DD + double, |x| >= |y| */
static inline dd_t ddadd_d2_d2_d(dd_t x, double y) {
  double s = x.x + y;
  return dd(s, ((x.x - s) + y) + x.y);
}
/* DD + double, any magnitudes */
static inline dd_t ddadd2_d2_d2_d(dd_t x, double y) {
  double s = x.x + y, v = s - x.x;
  return dd(s, ((x.x - (s - v)) + (y - v)) + x.y);
}
/* exact product of two doubles: s = RN(xy), lo = xy - s via fma */
static inline dd_t ddmul_d2_d_d(double x, double y) {
  double s = x * y;
  return dd(s, fma(x, y, -s));
}
/* DD * double: s = x.x*y, lo = x.y*y + (x.x*y - s) */
static inline dd_t ddmul_d2_d2_d(dd_t x, double y) {
  double s = x.x * y;
  return dd(s, fma(x.y, y, fma(x.x, y, -s)));
}
/* DD * DD: s = x.x*y.x, lo = x.x*y.y + x.y*y.x + (x.x*y.x - s) */
static inline dd_t ddmul_d2_d2_d2(dd_t x, dd_t y) {
  double s = x.x * y.x;
  return dd(s, fma(x.x, y.y, fma(x.y, y.x, fma(x.x, y.x, -s))));
}
/* DD squared: s = x.x^2, lo = 2 x.x x.y + (x.x^2 - s) */
static inline dd_t ddsqu_d2_d2(dd_t x) {
  double s = x.x * x.x;
  return dd(s, fma(x.x + x.x, x.y, fma(x.x, x.x, -s)));
}
/* DD times a power of two (exact) */
static inline dd_t ddscale_d2_d2_d(dd_t x, double s) { return dd(x.x * s, x.y * s); }
/* renormalize: FastTwoSum of head and tail */
static inline dd_t ddnormalize_d2_d2(dd_t x) {
  double s = x.x + x.y;
  return dd(s, (x.x - s) + x.y);
}
/* DD / DD with one division: t = 1/d.x, q = n.x t,
 * lo = t * ((n.x - q d.x) + n.y - q d.y) */
static inline dd_t dddiv_d2_d2_d2(dd_t n, dd_t d) {
  double t = 1.0 / d.x;
  double q = n.x * t;
  double r = fma(-q, d.x, n.x);
  r = fma(-q, d.y, r + n.y);
  return dd(q, r * t);
}
/* 1 / d as DD: t = 1/d, lo = t * (1 - t d) */
static inline dd_t ddrec_d2_d(double d) {
  double t = 1.0 / d;
  return dd(t, t * fma(-t, d, 1.0));
}
/* 1 / DD */
static inline dd_t ddrec_d2_d2(dd_t d) {
  double t = 1.0 / d.x;
  double r = fma(-t, d.x, 1.0);
  r = fma(-t, d.y, r);
  return dd(t, r * t);
}
/* sqrt of a DD: h = sqrt(d.x), lo = (d - h^2) / (2 h) using one division */
static inline dd_t ddsqrt_d2_d2(dd_t d) {
  double h = sqrt(d.x);
  double r = fma(-h, h, d.x) + d.y;
  return dd(h, r * (1.0 / (h + h)));
}

/* ---- float-float (FP32 analogues) ---- */
static inline ff_t ff(float h, float l) { ff_t r; r.x = h; r.y = l; return r; }
static inline ff_t ffadd_f2_f_f(float x, float y) { float s = x + y; return ff(s, (x - s) + y); }
static inline ff_t ffadd2_f2_f_f(float x, float y) {
  float s = x + y, v = s - x; return ff(s, (x - (s - v)) + (y - v));
}
static inline ff_t ffadd_f2_f2_f2(ff_t x, ff_t y) {
  float s = x.x + y.x; return ff(s, (((x.x - s) + y.x) + x.y) + y.y);
}
static inline ff_t ffadd2_f2_f2_f2(ff_t x, ff_t y) {
  float s = x.x + y.x, v = s - x.x; float e = (x.x - (s - v)) + (y.x - v);
  return ff(s, (e + x.y) + y.y);
}
static inline ff_t ffadd_f2_f_f2(float x, ff_t y) {
  float s = x + y.x; return ff(s, ((x - s) + y.x) + y.y);
}
static inline ff_t ffadd2_f2_f_f2(float x, ff_t y) {
  float s = x + y.x, v = s - x; return ff(s, ((x - (s - v)) + (y.x - v)) + y.y);
}
static inline ff_t ffadd_f2_f2_f(ff_t x, float y) {
  float s = x.x + y; return ff(s, ((x.x - s) + y) + x.y);
}
static inline ff_t ffadd2_f2_f2_f(ff_t x, float y) {
  float s = x.x + y, v = s - x.x; return ff(s, ((x.x - (s - v)) + (y - v)) + x.y);
}
static inline ff_t ffmul_f2_f_f(float x, float y) { float s = x * y; return ff(s, fmaf(x, y, -s)); }
static inline ff_t ffmul_f2_f2_f(ff_t x, float y) {
  float s = x.x * y; return ff(s, fmaf(x.y, y, fmaf(x.x, y, -s)));
}
static inline ff_t ffmul_f2_f2_f2(ff_t x, ff_t y) {
  float s = x.x * y.x; return ff(s, fmaf(x.x, y.y, fmaf(x.y, y.x, fmaf(x.x, y.x, -s))));
}
static inline ff_t ffsqu_f2_f2(ff_t x) {
  float s = x.x * x.x; return ff(s, fmaf(x.x + x.x, x.y, fmaf(x.x, x.x, -s)));
}
static inline ff_t ffscale_f2_f2_f(ff_t x, float s) { return ff(x.x * s, x.y * s); }
static inline ff_t ffnormalize_f2_f2(ff_t x) { float s = x.x + x.y; return ff(s, (x.x - s) + x.y); }
static inline ff_t ffdiv_f2_f2_f2(ff_t n, ff_t d) {
  float t = 1.0f / d.x, q = n.x * t;
  float r = fmaf(-q, d.x, n.x);
  r = fmaf(-q, d.y, r + n.y);
  return ff(q, r * t);
}
static inline ff_t ffrec_f2_f(float d) { float t = 1.0f / d; return ff(t, t * fmaf(-t, d, 1.0f)); }
/* 1 / FF */
static inline ff_t ffrec_f2_f2(ff_t d) {
  float t = 1.0f / d.x;
  float r = fmaf(-t, d.x, 1.0f);
  r = fmaf(-t, d.y, r);
  return ff(t, r * t);
}
static inline ff_t ffsqrt_f2_f2(ff_t d) {
  float h = sqrtf(d.x);
  float r = fmaf(-h, h, d.x) + d.y;
  return ff(h, r / (h + h));
}

#endif
