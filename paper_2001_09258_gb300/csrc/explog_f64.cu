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
#include "sleefcu_common.cuh"

namespace sleefcu {
namespace explog64 {

constexpr double R_LN2 = 0x1.71547652b82fep0;
constexpr double L2A = 0x1.62e42fefa39efp-1;
constexpr double L2B = 0x1.abc9e3b39803fp-56;
constexpr double L2H = 0x1.62e42fefa3800p-1;   // 42 bits: e*L2H exact for |e| < 2^11
constexpr double L2L = 0x1.ef35793c76730p-45;
constexpr uint64_t B746 = 0x4087500000000000ull;  // bits of 746.0
constexpr uint64_t DMAX = 0x7FEFFFFFFFFFFFFFull;
constexpr uint64_t INF = 0x7FF0000000000000ull;

static __constant__ double kExpU10[11] = {
  0x1.0000000000000p-1, 0x1.555555555555bp-3, 0x1.5555555555503p-5, 0x1.111111110ec3fp-7,
  0x1.6c16c16c305dap-10, 0x1.a01a01b38a1ccp-13, 0x1.a01a01364ed77p-16, 0x1.71ddf0027528ep-19,
  0x1.27e5b4917ffe5p-22, 0x1.af6c1dcd03fd7p-26, 0x1.1e3d09ab8b9a5p-29};
static __constant__ double kExpU35[9] = {
  0x1.ffffffffffed1p-2, 0x1.5555555550776p-3, 0x1.5555555589411p-5, 0x1.11111125c3b1dp-7,
  0x1.6c16c0c7b3762p-10, 0x1.a0198d1cfb5cfp-13, 0x1.a01b7d10e56f2p-16, 0x1.72e95f1b1c6d2p-19,
  0x1.27076dd8a5103p-22};
static __constant__ double kLogU10[8] = {
  0x1.555555555554fp-4, 0x1.999999999c179p-7, 0x1.24924921e457cp-9, 0x1.c71c748fb0e5ep-12,
  0x1.745c4adfd4929p-14, 0x1.3b35c02f141cfp-16, 0x1.0dcba14fc06c7p-18, 0x1.1b8139759f314p-20};
static __constant__ double kLogU35[7] = {
  0x1.5555555555775p-4, 0x1.99999998f0e71p-7, 0x1.249249b213a2dp-9, 0x1.c71c01680d46ap-12,
  0x1.7474e2e4fcac3p-14, 0x1.3852c703d6843p-16, 0x1.3abef8cc48463p-18};
constexpr double PL_C1H = 0x1.5555555555555p-4, PL_C1L = 0x1.54855a03b34d8p-58;
static __constant__ double kPowLog[9] = {
  0x1.999999999999cp-7, 0x1.2492492492062p-9, 0x1.c71c71c78a1b0p-12, 0x1.745d171399b86p-14,
  0x1.3b13bf3c5b892p-16, 0x1.110e98ef52765p-18, 0x1.e26f3be0efb86p-21, 0x1.a57c235e7b51bp-23,
  0x1.e37c78d194e20p-25};
static __constant__ double kPowExp[10] = {
  0x1.555555555555ap-3, 0x1.5555555555498p-5, 0x1.111111110f0acp-7, 0x1.6c16c16c4d9f3p-10,
  0x1.a01a01b2b4f71p-13, 0x1.a01a010b94555p-16, 0x1.71ddf039a6182p-19, 0x1.27e54bd4df84bp-22,
  0x1.af6e560a2694ap-26, 0x1.1fda157dfad50p-29};

// value of an integer-valued double with |k| < 2^31, on the integer pipe
__device__ __forceinline__ int int_of(double k) {
  uint64_t b = bits(k);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  int v = e < 0 ? 0 : (int)(m >> (52 - e));
  return (b >> 63) ? -v : v;
}
// exact double of an int with |v| < 2^31, on the integer pipe
__device__ __forceinline__ double dbl_of(int v) {
  if (v == 0) return 0.0;
  uint32_t a = v < 0 ? (uint32_t)(-v) : (uint32_t)v;
  int p = 31 - __clz(a);                         // a in [2^p, 2^(p+1))
  uint64_t m = ((uint64_t)a << (52 - p)) & 0x000FFFFFFFFFFFFFull;
  return from_bits(((uint64_t)(v < 0) << 63) | ((uint64_t)(p + 1023) << 52) | m);
}
__device__ __forceinline__ double pow2i(int k) { return from_bits((uint64_t)(k + 1023) << 52); }

// y * 2^k for y in [0.5, 2): exponent-field add when the result is normal,
// otherwise two multiplications by normal powers of two (rounds once)
__device__ __forceinline__ double scale2(double y, int k) {
  if (k >= -1021 && k <= 1023) return from_bits(bits(y) + ((uint64_t)(int64_t)k << 52));
  int k1 = k / 2, k2 = k - k1;
  return __dmul_rn(__dmul_rn(y, pow2i(k1)), pow2i(k2));
}

template <int N>
__device__ __forceinline__ double exp_core(double x, const double (&c)[N]) {
  uint64_t b = bits(x), ab = b & ABS64;
  bool inr = ab <= B746;
  double xc = inr ? x : 0.0;
  double k = rint(__dmul_rn(xc, R_LN2));
  double r = __fma_rn(k, -L2A, xc);
  r = __fma_rn(k, -L2B, r);
  double s = __dmul_rn(r, r);
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
  double k = rint(__dmul_rn(xc, R_LN2));
  double h = __fma_rn(k, -L2A, xc);
  double r = __fma_rn(k, -L2B, h);
  double rl = __fma_rn(k, -L2B, __dsub_rn(h, r));
  double s = __dmul_rn(r, r);
  double w = __fma_rn(s, poly(r, kExpU10), rl);
  d2 o = add_dd_fast(1.0, r);
  double y = scale2(__dadd_rn(o.x, __dadd_rn(o.y, w)), int_of(k));
  if (!inr) y = is_nan_b(b) ? from_bits(QNAN64) : ((b >> 63) ? 0.0 : from_bits(INF));
  return canon(y);
}
struct ExpU10 { __device__ double operator()(double x) const { return exp_core_u10(x); } };
struct ExpU35 { __device__ double operator()(double x) const { return exp_core(x, kExpU35); } };

// a = bits of a finite positive double: m in [0.75, 1.5) and e with a = m 2^e
__device__ __forceinline__ double log_reduce(uint64_t a, int &e) {
  int off = 0;
  if (a < 0x0010000000000000ull) {                // subnormal: scale by 2^64 (exact)
    a = bits(__dmul_rn(from_bits(a), 0x1p64));
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
    d2 z = div_d2d2(D2(__dmul_rn(2.0, __dsub_rn(m, 1.0)), 0.0), den);
    double t = __dmul_rn(z.x, z.x);
    double corr = __dmul_rn(__dmul_rn(z.x, t), poly(t, kLogU10));
    double ed = dbl_of(e);
    d2 r = add_d2d2_fast(D2(__dmul_rn(ed, L2H), __dmul_rn(ed, L2L)), z);
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
    double z = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(m, 1.0)), __dadd_rn(1.0, m));
    double t = __dmul_rn(z, z);
    double lm = __fma_rn(__dmul_rn(z, t), poly(t, kLogU35), z);
    return canon(log_special(b, __fma_rn(dbl_of(e), L2A, lm)));
  }
};

// ---- pow ----
__device__ __forceinline__ d2 logk(uint64_t a) {
  int e;
  double m = log_reduce(a, e);
  d2 den = add_dd_fast(1.0, m);
  d2 z = div_d2d2(D2(__dmul_rn(2.0, __dsub_rn(m, 1.0)), 0.0), den);
  d2 t = sqr_d2(z);
  double q = poly(t.x, kPowLog);
  d2 w = add_d2_d_fast(D2(PL_C1H, PL_C1L), __dmul_rn(t.x, q));
  w = mul_d2d2(t, w);
  w = mul_d2d2(z, w);
  d2 lm = add_d2d2_fast(z, w);
  double ed = dbl_of(e);
  return add_d2d2_fast(D2(__dmul_rn(ed, L2H), __dmul_rn(ed, L2L)), lm);
}
__device__ __forceinline__ double expk(d2 Y) {
  bool inr = (bits(Y.x) & ABS64) <= B746;
  double yh = inr ? Y.x : 0.0, yl = inr ? Y.y : 0.0;
  double k = rint(__dmul_rn(yh, R_LN2));
  double u = __fma_rn(k, -L2A, yh);
  d2 r = add_dd(u, __fma_rn(k, -L2B, yl));
  d2 q = scale_d2(sqr_d2(r), 0.5);
  double p = poly(r.x, kPowExp);
  double v = __dmul_rn(__dmul_rn(__dmul_rn(r.x, r.x), r.x), p);
  d2 s = add_d2d2(r, q);
  s = add_d2_d(s, v);
  s = add_d_d2_fast(1.0, s);
  double y = scale2(__dadd_rn(s.x, s.y), int_of(k));
  if (!inr) y = (bits(Y.x) >> 63) ? 0.0 : from_bits(INF);
  return y;
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
    bool yint = yfin && (y == trunc(y));
    bool yodd = yint && ay < 0x4340000000000000ull && (((uint64_t)(int64_t)y) & 1);   // |y| < 2^53
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
UNARY64(exp_u10_f64, ExpU10)
UNARY64(exp_u35_f64, ExpU35)
UNARY64(log_u10_f64, LogU10)
UNARY64(log_u35_f64, LogU35)

extern "C" sleefcu_status sleefcu_pow_u10_f64(const double *x, const double *y, double *out, size_t n,
                                              sleefcu_stream s) {
  return launch_binary64<explog64::PowU10>("sleefcu_pow_u10_f64", x, y, out, n, s);
}
extern "C" sleefcu_status sleefcu_pow_u35_f64(const double *x, const double *y, double *out, size_t n,
                                              sleefcu_stream s) {
  return launch_binary64<explog64::PowU10>("sleefcu_pow_u35_f64", x, y, out, n, s);
}
#undef UNARY64
#endif  // SLEEFCU_FUNCTORS_ONLY
