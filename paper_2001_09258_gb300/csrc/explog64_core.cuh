// Shared FP64 exp/log cores: constants, coefficient tables and the reduction
// and reconstruction steps used by exp/log/pow and by the functions built on
// them (exp2, exp10, expm1, log2, log10, log1p, hyperbolics and their
// inverses).  Sections 5.5-5.7 of the paper; the DD arithmetic of Section 3.
#pragma once
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
  return dmul(dmul(y, pow2i(k1)), pow2i(k2));
}

// 2^k for k in [-1074, 1023], normal or subnormal, from the bits
__device__ __forceinline__ double pow2_any(int k) {
  return k >= -1022 ? pow2i(k) : from_bits(1ull << (k + 1074));
}

// a DD with a normal positive head, scaled by 2^-ex (ex its head's
// exponent): the head's significand in [1, 2) is taken from the bits, the
// tail (possibly zero or subnormal) is multiplied; then halved if the head
// is >= 1.5 (ex incremented).  Same values as scaling both parts by
// multiplications, one or two FP64 operations fewer.
__device__ __forceinline__ d2 log_mantissa(d2 a, int &ex) {
  ex = (int)(bits(a.x) >> 52) - 1023;
  uint64_t hb = (bits(a.x) & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
  double t = dmul(a.y, pow2_any(-ex));
  if (hb >= 0x3FF8000000000000ull) {
    hb -= 0x0010000000000000ull;
    t = dmul(t, 0.5);
    ex++;
  }
  return D2(from_bits(hb), t);
}

// 2^k (1 + r + rl) with the 1-ULP polynomial, |r| <= ln2/2: the residual rl
// joins the polynomial part and 1 + r is a DD, so the last addition is the
// only rounding of order one ulp (Section 5.6)
__device__ __forceinline__ double exp_tail_u10(double r, double rl, int k) {
  double s = dmul(r, r);
  double w = __fma_rn(s, poly(r, kExpU10), rl);
  d2 o = add_dd_fast(1.0, r);
  return scale2(__dadd_rn(o.x, __dadd_rn(o.y, w)), k);
}

// For |Y.x| <= 746: k = rint(Y.x/ln2) and e^(Y - k ln2) - 1 as a DD.  The
// head Y.x - k L2A is exact (k has at most 11 bits and the result is below
// 1/2), so the reduced argument is a DD to about 2^-100.
__device__ __forceinline__ d2 expk_s(d2 Y, double &k) {
  k = drint(dmul(Y.x, R_LN2));
  double u = __fma_rn(k, -L2A, Y.x);
  d2 r = add_dd(u, __fma_rn(k, -L2B, Y.y));
  d2 q = scale_d2(sqr_d2(r), 0.5);
  double p = poly(r.x, kPowExp);
  double v = dmul(dmul(dmul(r.x, r.x), r.x), p);
  d2 s = add_d2d2(r, q);
  return add_d2_d(s, v);
}

// e^Y for a DD Y (the exponential inside pow, Section 5.7): overflow to
// +inf, underflow with subnormals rounded once
__device__ __forceinline__ double expk(d2 Y) {
  bool inr = (bits(Y.x) & ABS64) <= B746;
  double yh = inr ? Y.x : 0.0, yl = inr ? Y.y : 0.0;
  double k;
  d2 s = expk_s(D2(yh, yl), k);
  s = add_d_d2_fast(1.0, s);
  double y = scale2(__dadd_rn(s.x, s.y), int_of(k));
  if (!inr) y = (bits(Y.x) >> 63) ? 0.0 : from_bits(INF);
  return y;
}

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

// log of a DD a > 0 with a finite head: a = m 2^e, m in [0.75, 1.5) (heads
// below DBL_MIN scaled by 2^64 first); returns log m = z + z^3 P(z^2) as a DD
// with z = 2(m-1)/(m+1) in DD (Section 5.5 on a DD argument)
__device__ __forceinline__ d2 logm_u10(d2 a, int &e) {
  int off = 0;
  if (lt_c(a.x, 0x1p-1022)) { a = scale_d2(a, 0x1p64); off = 64; }
  int ex;
  d2 m = log_mantissa(a, ex);
  d2 num = scale_d2(add_dd(__dsub_rn(m.x, 1.0), m.y), 2.0);
  d2 den = add_d_d2(1.0, m);
  d2 z = div_d2d2(num, den);
  double t = dmul(z.x, z.x);
  double corr = dmul(dmul(z.x, t), poly(t, kLogU10));
  e = ex - off;
  return add_d2_d_fast(z, corr);
}

// the same in double for the 3.5-ULP forms (z rounded once)
__device__ __forceinline__ double logm_u35(d2 a, int &e) {
  int off = 0;
  if (lt_c(a.x, 0x1p-1022)) { a = scale_d2(a, 0x1p64); off = 64; }
  int ex;
  d2 m = log_mantissa(a, ex);
  double num = dmul(2.0, __dadd_rn(__dsub_rn(m.x, 1.0), m.y));
  double z = dmul(num, __ddiv_rn(1.0, __dadd_rn(1.0, m.x)));
  double t = dmul(z, z);
  e = ex - off;
  return __fma_rn(dmul(z, t), poly(t, kLogU35), z);
}

// log m in double with z = 2(m-1)/(m+1) corrected once: the residual
// num - z (1 + m) (the rounding of 1 + m and the DD tail of m included) goes
// back through the reciprocal, then the 3.5-ULP polynomial; for the 3.5-ULP
// forms whose logarithm is small against the rounding of its argument
// (asinh, acosh, atanh)
__device__ __forceinline__ double logm_u20(d2 a, int &e) {
  int off = 0;
  if (lt_c(a.x, 0x1p-1022)) { a = scale_d2(a, 0x1p64); off = 64; }
  int ex;
  d2 m = log_mantissa(a, ex);
  double num = dmul(2.0, __dadd_rn(__dsub_rn(m.x, 1.0), m.y));
  double den = __dadd_rn(1.0, m.x);
  double rd = __ddiv_rn(1.0, den);
  double z = dmul(num, rd);
  double r = __dsub_rn(__fma_rn(-z, den, num), dmul(z, __dadd_rn(__dadd_rn(__dsub_rn(1.0, den), m.x), m.y)));
  z = __fma_rn(r, rd, z);
  double t = dmul(z, z);
  e = ex - off;
  return __fma_rn(dmul(z, t), poly(t, kLogU35), z);
}

// log of a DD y > 0 with the 11-term DD polynomial of pow's logarithm
// (about 2^-66 relative): m in [0.75, 1.5) from the head, z = 2(m-1)/(m+1)
// in DD
__device__ __forceinline__ d2 logk_dd(d2 y) {
  int off = 0;
  if (lt_c(y.x, 0x1p-1022)) { y = scale_d2(y, 0x1p64); off = 64; }
  int ex;
  d2 m = log_mantissa(y, ex);
  d2 num = scale_d2(add_dd(__dsub_rn(m.x, 1.0), m.y), 2.0);
  d2 z = div_d2d2(num, add_d_d2(1.0, m));
  d2 t = sqr_d2(z);
  double q = poly(t.x, kPowLog);
  d2 w = add_d2_d_fast(D2(PL_C1H, PL_C1L), dmul(t.x, q));
  w = mul_d2d2(t, w);
  w = mul_d2d2(z, w);
  d2 lm = add_d2d2_fast(z, w);
  double ed = dbl_of(ex - off);
  return add_d2d2(D2(dmul(ed, L2H), dmul(ed, L2L)), lm);
}

}  // namespace explog64
}  // namespace sleefcu
