// FP64 pow (u10; the u35 entry point runs the same kernel) for sm_103a.
//
// pow (Section 5.7): exp(y log|x|) with an 11-term DD logarithm, the product
//   in DD and a 13-term exponential whose leading terms are DD; C99 Annex F
//   special pairs are selected last (Section 5.10).
//
// Multiplications run in software on the integer pipe through one
// out-of-line copy of the exact multiply (SLEEFCU_SOFT_MUL 2 for this
// translation unit): measured on GB300 on the full-set workload, 1.085x the
// form inlined at every call site.  Same bits either way.
#ifndef SLEEFCU_FUNCTORS_ONLY
#define SLEEFCU_SOFT_MUL 2
#endif
#include "explog64_core.cuh"

namespace sleefcu {
namespace explog64 {

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
#endif  // SLEEFCU_FUNCTORS_ONLY
