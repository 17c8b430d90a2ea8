// FP64 exp and log (u10 and u35) for sm_103a (pow: pow_f64.cu).
//
// exp (Section 5.6): k = rint(x/ln2), r = x - k ln2 by two fma steps, one
//   13-term (u10) or 11-term (u35) polynomial without DD, reconstruction by
//   adding k to the exponent field (integer pipe) when the result is normal,
//   else by two multiplications that round once.
// log (Section 5.5): subnormals scaled by 2^64; e and m in [0.75, 1.5) taken
//   from the exponent and significand bits; z = 2(m-1)/(m+1) in DD;
//   log m = z + z^3 P(z^2); e ln2 + log m in DD.
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

#undef UNARY64
#undef UNARY64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
