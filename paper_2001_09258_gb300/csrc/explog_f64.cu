// FP64 exp, log, pow (u10 and u35) for sm_103a.
//
// exp (Section 5.6): k = rint(x/ln2), r = x - k ln2 by two fma steps, one
//   13-term (u10) or 11-term (u35) polynomial without DD, reconstruction by
//   adding k to the exponent field (integer pipe) when the result is normal,
//   else by two multiplications that round once.
// log (Section 5.5): subnormals scaled by 2^64; e and m in [0.75, 1.5) taken
//   from the exponent and significand bits; z = 2(m-1)/(m+1) in DD;
//   log m = z + z^3 P(z^2); e ln2 + log m in DD.
// pow (Section 5.7): exp(y log|x|) with an 11-term DD logarithm, the product
//   in DD and a 13-term exponential whose leading terms are DD; C99 Annex F
//   special pairs are selected last (Section 5.10).
#include "explog64_core.cuh"

namespace sleefcu {
namespace explog64 {

template <int N>
__device__ __forceinline__ double exp_core(double x, const double (&c)[N]) {
  uint64_t b = bits(x), ab = b & ABS64;
  bool inr = ab <= B746;
  double xc = inr ? x : 0.0;
  double k = drint(dmul(xc, R_LN2));
  double r = __fma_rn(k, -L2A, xc);
  r = __fma_rn(k, -L2B, r);
  double s = dmul(r, r);
  double v = __fma_rn(s, poly(r, c), r);
  double y = scale2(__dadd_rn(1.0, v), int_of(k));
  if (!inr) y = is_nan_b(b) ? from_bits(QNAN64) : ((b >> 63) ? 0.0 : from_bits(INF));
  return canon(y);
}
// u10: keeps the residual of r = h - k L2B and forms 1 + r as a DD
__device__ __forceinline__ double exp_core_u10(double x) {
  uint64_t b = bits(x), ab = b & ABS64;
  bool inr = ab <= B746;
  double xc = inr ? x : 0.0;
  double k = drint(dmul(xc, R_LN2));
  double h = __fma_rn(k, -L2A, xc);
  double r = __fma_rn(k, -L2B, h);
  double rl = __fma_rn(k, -L2B, __dsub_rn(h, r));
  double y = exp_tail_u10(r, rl, int_of(k));
  if (!inr) y = is_nan_b(b) ? from_bits(QNAN64) : ((b >> 63) ? 0.0 : from_bits(INF));
  return canon(y);
}
struct ExpU10 { __device__ double operator()(double x) const { return exp_core_u10(x); } };
struct ExpU35 { __device__ double operator()(double x) const { return exp_core(x, kExpU35); } };

// a = bits of a finite positive double: m in [0.75, 1.5) and e with a = m 2^e
__device__ __forceinline__ double log_reduce(uint64_t a, int &e) {
  int off = 0;
  if (a < 0x0010000000000000ull) {                // subnormal: scale by 2^64 (exact)
    a = bits(dmul(from_bits(a), 0x1p64));
    off = 64;
  }
  int ex = (int)(a >> 52) - 1023;
  uint64_t mb = (a & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;   // significand in [1, 2)
  if (mb & 0x0008000000000000ull) { mb -= 0x0010000000000000ull; ex++; } // >= 1.5: halve
  e = ex - off;
  return from_bits(mb);
}
__device__ __forceinline__ double log_special(uint64_t b, double y) {
  if ((b & ABS64) == 0) return from_bits(0xFFF0000000000000ull);   // log(+-0) = -inf
  if ((b >> 63) || is_nan_b(b)) return from_bits(QNAN64);
  if (b == INF) return from_bits(INF);
  return y;
}

struct LogU10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    uint64_t a = (b - 1) < DMAX ? b : 0x3FF0000000000000ull;
    int e;
    double m = log_reduce(a, e);
    d2 den = add_dd_fast(1.0, m);
    d2 z = div_d2d2(D2(dmul(2.0, __dsub_rn(m, 1.0)), 0.0), den);
    double t = dmul(z.x, z.x);
    double corr = dmul(dmul(z.x, t), poly(t, kLogU10));
    double ed = dbl_of(e);
    d2 r = add_d2d2_fast(D2(dmul(ed, L2H), dmul(ed, L2L)), z);
    r = add_d2_d_fast(r, corr);
    return canon(log_special(b, __dadd_rn(r.x, r.y)));
  }
};
struct LogU35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    uint64_t a = (b - 1) < DMAX ? b : 0x3FF0000000000000ull;
    int e;
    double m = log_reduce(a, e);
    double z = dmul(dmul(2.0, __dsub_rn(m, 1.0)), __ddiv_rn(1.0, __dadd_rn(1.0, m)));
    double t = dmul(z, z);
    double lm = __fma_rn(dmul(z, t), poly(t, kLogU35), z);
    return canon(log_special(b, __fma_rn(dbl_of(e), L2A, lm)));
  }
};

// ---- pow ----
__device__ __forceinline__ d2 logk(uint64_t a) {
  int e;
  double m = log_reduce(a, e);
  d2 den = add_dd_fast(1.0, m);
  d2 z = div_d2d2(D2(dmul(2.0, __dsub_rn(m, 1.0)), 0.0), den);
  d2 t = sqr_d2(z);
  double q = poly(t.x, kPowLog);
  d2 w = add_d2_d_fast(D2(PL_C1H, PL_C1L), dmul(t.x, q));
  w = mul_d2d2(t, w);
  w = mul_d2d2(z, w);
  d2 lm = add_d2d2_fast(z, w);
  double ed = dbl_of(e);
  return add_d2d2_fast(D2(dmul(ed, L2H), dmul(ed, L2L)), lm);
}

struct PowU10 {
  __device__ double operator()(double x, double y) const {
    uint64_t bx = bits(x), by = bits(y);
    uint64_t ax = bx & ABS64, ay = by & ABS64;
    bool xfin = ax < INF, yfin = ay < INF;
    bool xnan = ax > INF, ynan = ay > INF;
    bool xneg = (bx >> 63) && ax != 0 && !xnan;    // x < 0
    uint64_t a = (ax - 1) < DMAX ? ax : 0x3FF0000000000000ull;
    double yc = yfin ? y : 0.0;
    bool yint = yfin && integral_b(ay);
    bool yodd = yfin && odd_int_b(ay);
    double r = expk(mul_d2_d(logk(a), yc));
    if (xneg && yodd) r = -r;
    if (xneg && xfin && yfin && !yint) r = from_bits(QNAN64);
    bool yneg = (by >> 63) && ay != 0 && !ynan;    // y < 0
    if (ax == 0 && ay != 0 && !ynan) {
      if (yneg) r = yodd ? neg_if(from_bits(INF), (bx >> 63) != 0) : from_bits(INF);
      else r = yodd ? x : 0.0;
    }
    if (ay == INF) {
      if (ax == 0x3FF0000000000000ull) r = 1.0;
      else r = ((ax < 0x3FF0000000000000ull) == yneg) ? from_bits(INF) : 0.0;
    }
    if (ax == INF) {
      if (!(bx >> 63)) r = yneg ? 0.0 : from_bits(INF);
      else if (yneg) r = yodd ? -0.0 : 0.0;
      else r = yodd ? from_bits(0xFFF0000000000000ull) : from_bits(INF);
    }
    if (xnan || ynan) r = from_bits(QNAN64);
    if (ay == 0 || bx == 0x3FF0000000000000ull) r = 1.0;
    return canon(r);
  }
};

}  // namespace explog64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define UNARY64(NAME, F)                                                                    \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_unary64<explog64::F>("sleefcu_" #NAME, x, out, n, s);                     \
  }
#define UNARY64_MASKED(NAME, F)                                                     \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<explog64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
UNARY64(exp_u10_f64, ExpU10)
UNARY64_MASKED(exp_u10_f64, ExpU10)
UNARY64(exp_u35_f64, ExpU35)
UNARY64_MASKED(exp_u35_f64, ExpU35)
UNARY64(log_u10_f64, LogU10)
UNARY64_MASKED(log_u10_f64, LogU10)
UNARY64(log_u35_f64, LogU35)
UNARY64_MASKED(log_u35_f64, LogU35)

extern "C" sleefcu_status sleefcu_pow_u10_f64(const double *x, const double *y, double *out, size_t n,
                                              sleefcu_stream s) {
  return launch_binary64<explog64::PowU10>("sleefcu_pow_u10_f64", x, y, out, n, s);
}
extern "C" sleefcu_status sleefcu_pow_u35_f64(const double *x, const double *y, double *out, size_t n,
                                              sleefcu_stream s) {
  return launch_binary64<explog64::PowU10>("sleefcu_pow_u35_f64", x, y, out, n, s);
}
extern "C" sleefcu_status sleefcu_pow_u10_f64_masked(const double *x, const double *y, const uint8_t *mask,
                                                     double *out, size_t n, sleefcu_stream s) {
  return launch_masked64b<explog64::PowU10>("sleefcu_pow_u10_f64_masked", x, y, mask, out, n, s);
}
extern "C" sleefcu_status sleefcu_pow_u35_f64_masked(const double *x, const double *y, const uint8_t *mask,
                                                     double *out, size_t n, sleefcu_stream s) {
  return launch_masked64b<explog64::PowU10>("sleefcu_pow_u35_f64_masked", x, y, mask, out, n, s);
}
#undef UNARY64
#undef UNARY64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
