/*
 * Shared helpers of the oracle (scalar C, test infrastructure only: only
 * tests/, the smoke check and the CPU-baseline leg of the benchmark use
 * anything under oracle/).
 */
#ifndef ORACLE_COMMON_H
#define ORACLE_COMMON_H
#include <stdint.h>
#include <string.h>
#include <math.h>
#include "dd.h"

/* Every NaN result is the canonical quiet NaN with a clear sign bit, chosen
 * by an explicit select at the end of each function (reading of Section 5.10:
 * the paper does not fix NaN payloads). */
static inline double canon_nan(void) { uint64_t b = 0x7FF8000000000000ULL; double d; memcpy(&d, &b, 8); return d; }
static inline float canon_nanf(void) { uint32_t b = 0x7FC00000U; float f; memcpy(&f, &b, 4); return f; }
static inline double canon(double y) { return isnan(y) ? canon_nan() : y; }
static inline float canonf(float y) { return isnan(y) ? canon_nanf() : y; }
static inline uint64_t dbits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static inline uint32_t fbits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* n mod 4 (two's complement sense) of an integer-valued double or float n,
 * read from its bits: n = m 2^e with the integer significand m */
static inline int low2_of_integral(double n) {
  uint64_t b = dbits(n);
  int be = (int)((b >> 52) & 0x7FF), e = be - 1075;
  uint64_t m = (b & 0x000FFFFFFFFFFFFFULL) | 0x0010000000000000ULL;
  int v = (be == 0 || e >= 2 || e < -52) ? 0 : (int)((e >= 0 ? m << e : m >> -e) & 3);
  return (b >> 63) ? (4 - v) & 3 : v;
}
static inline int low2_of_integralf(float n) {
  uint32_t b = fbits(n);
  int be = (int)((b >> 23) & 0xFF), e = be - 150;
  uint32_t m = (b & 0x007FFFFFU) | 0x00800000U;
  int v = (be == 0 || e >= 2 || e < -23) ? 0 : (int)((e >= 0 ? m << e : m >> -e) & 3);
  return (b >> 31) ? (4 - v) & 3 : v;
}

/* Estrin's scheme (Section 5, polynomial evaluation): with pw[k] = t^(2^k),
 * E(c, n) = c[0] for n = 1, else fma(t^m, E(c+m, n-m), E(c, m)) where m is
 * the largest power of two below n.  The same tree is used for every
 * polynomial of the library so that both implementations agree bit for bit. */
static inline double estrin_d(const double *c, int n, const double *pw) {
  if (n == 1) return c[0];
  int m = 1, k = 0;
  while (2 * m < n) { m *= 2; k++; }
  return fma(pw[k], estrin_d(c + m, n - m, pw), estrin_d(c, m, pw));
}
static inline float estrin_f(const float *c, int n, const float *pw) {
  if (n == 1) return c[0];
  int m = 1, k = 0;
  while (2 * m < n) { m *= 2; k++; }
  return fmaf(pw[k], estrin_f(c + m, n - m, pw), estrin_f(c, m, pw));
}
/* evaluate an n-coefficient polynomial in t (c[0] is the constant term) */
/* (only the powers t^(2^k) with 2^k < n are formed: the tree uses no other) */
static inline double poly_d(double t, const double *c, int n) {
  double pw[5];
  pw[0] = t;
  for (int k = 1; k < 5 && (1 << k) < n; k++) pw[k] = pw[k - 1] * pw[k - 1];
  return estrin_d(c, n, pw);
}
static inline float poly_f(float t, const float *c, int n) {
  float pw[5];
  pw[0] = t;
  for (int k = 1; k < 5 && (1 << k) < n; k++) pw[k] = pw[k - 1] * pw[k - 1];
  return estrin_f(c, n, pw);
}

/* Payne-Hanek reduction, FP64 (phtab.c / trig64.c) */
dd_t oracle_ph_reduce_dd(double d, int *q);

#endif
