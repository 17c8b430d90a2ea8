// The remaining C99 real functions, binary64 and binary32, for sm_103a.
//
// Exact functions (C99 7.12 and Annex F): fabs, copysign, fmax, fmin, fdim,
// trunc, floor, ceil, round, rint, nextafter, logb, ilogb, ldexp, frexp, modf.
// binary64 trunc, floor, ceil, rint, round and modf round on the integer
// pipe (binary32 uses the hardware's roundToIntegral operations, which cost
// little there); everything that reads or builds an exponent (logb, ilogb,
// ldexp, frexp) and every comparison runs on the integer pipe.  ldexp splits
// x into m 2^e with m in [1, 2) and either writes the exponent field (normal
// results) or rounds m 2^(e + n + 1074) to an integer once (subnormal
// results).  Every NaN result is the canonical quiet NaN (fabs and copysign
// included).  Choices C99 leaves open:
// fmax(+0, -0) = +0, fmin(+0, -0) = -0, ilogb(0) = INT_MIN, ilogb(NaN) =
// INT_MAX, frexp(inf or NaN) stores 0.
//
// Approximated functions (0.5-ULP and 3.5-ULP forms):
//   sqrt   the IEEE square root (both forms: the correctly rounded hardware
//          sequence costs less than any 3.5-ULP one on this chip)
//   hypot  the larger magnitude's exponent e taken out exactly (the operands
//          times 2^-e, one rounding at most), the sum of squares and its square
//          root in DD (FF) arithmetic (u05) or one fma and a square root
//          (u35), then times 2^e
//   sinpi, cospi  x = q/2 + s exactly (q = rint(2x), |s| <= 1/4); the
//          quadrant's parity selects the coefficients of one polynomial shape,
//          sin(pi s) = s P(t) or cos(pi s) = 1 + t P(t), t = s^2, with no
//          divergent branch (Section 5's evaluation); three DD (FF) Horner
//          steps in the u05 forms
//
// All kernels are grid-stride with 16-byte accesses; the functions are
// memory bound except the u05 forms of hypot, sinpi and cospi.
#include <climits>
#include "sleefcu_common.cuh"
#include "sleefcu_dd.cuh"

namespace sleefcu {
namespace c99 {

constexpr uint64_t SIGN64 = 0x8000000000000000ull, FRAC64 = 0x000FFFFFFFFFFFFFull;
constexpr uint32_t SIGN32 = 0x80000000u, FRAC32 = 0x007FFFFFu;

// The bits of a double or float through an opaque register move: the
// compiler may turn a NaN or infinity test written on the bits back into a
// floating-point comparison, which takes an FP64-pipe slot on this chip.
__device__ __forceinline__ uint64_t ib(double d) {
  uint64_t r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(d));
  return r;
}
__device__ __forceinline__ uint32_t ibf(float f) {
  uint32_t r;
  asm("mov.b32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}
__device__ __forceinline__ double canon_i(double y) { return (ib(y) & ABS64) > EXP64 ? from_bits(QNAN64) : y; }
__device__ __forceinline__ float canonf_i(float y) { return (ibf(y) & ABS32) > EXP32 ? from_fbits(QNAN32) : y; }

// ---------------- exponent handling on the integer pipe ----------------
// finite non-zero |x| (its bits ab) = m 2^e, m in [1, 2)
__device__ __forceinline__ int expo64(uint64_t ab) {
  int E = (int)(ab >> 52);
  return E ? E - 1023 : -1011 - __clzll((long long)ab);
}
__device__ __forceinline__ uint64_t mant64(uint64_t ab) {   // the bits of m
  int E = (int)(ab >> 52);
  uint64_t f = E ? ab : ab << (__clzll((long long)ab) - 11);
  return (f & FRAC64) | 0x3FF0000000000000ull;
}
__device__ __forceinline__ int expo32(uint32_t ab) {
  int E = (int)(ab >> 23);
  return E ? E - 127 : -118 - __clz((int)ab);
}
__device__ __forceinline__ uint32_t mant32(uint32_t ab) {
  int E = (int)(ab >> 23);
  uint32_t f = E ? ab : ab << (__clz((int)ab) - 8);
  return (f & FRAC32) | 0x3F800000u;
}
// 2^k exactly: k in [-1074, 1023] (binary64), [-149, 127] (binary32)
__device__ __forceinline__ double pow2_64(int k) {
  return k >= -1022 ? from_bits((uint64_t)(k + 1023) << 52) : from_bits(1ull << (k + 1074));
}
__device__ __forceinline__ float pow2_32(int k) {
  return k >= -126 ? from_fbits((uint32_t)(k + 127) << 23) : from_fbits(1u << (k + 149));
}

__device__ __forceinline__ double ldexp64(double x, int n) {
  uint64_t b = ib(x), ab = b & ABS64, sg = b & SIGN64;
  if (ab == 0 || ab >= EXP64) return canon_i(x);
  n = max(min(n, 4000), -4000);
  int k = expo64(ab) + n;
  uint64_t mb = mant64(ab);
  if (k > 1023) return from_bits(sg | EXP64);
  if (k >= -1022) return from_bits(sg | (mb + ((uint64_t)(long long)k << 52)));
  int kk = k + 1074;                                        // subnormal: one rounding on the 2^-1074 grid
  if (kk < -1) return from_bits(sg);
  double r = dmul(drint(dmul(from_bits(mb), pow2_64(kk))), 0x1p-1074);
  return from_bits(sg | ib(r));
}
__device__ __forceinline__ float ldexp32(float x, int n) {
  uint32_t b = ibf(x), ab = b & ABS32, sg = b & SIGN32;
  if (ab == 0 || ab >= EXP32) return canonf_i(x);
  n = max(min(n, 1000), -1000);
  int k = expo32(ab) + n;
  uint32_t mb = mant32(ab);
  if (k > 127) return from_fbits(sg | EXP32);
  if (k >= -126) return from_fbits(sg | (mb + ((uint32_t)k << 23)));
  int kk = k + 149;
  if (kk < -1) return from_fbits(sg);
  float r = __fmul_rn(rintf(__fmul_rn(from_fbits(mb), pow2_32(kk))), 0x1p-149f);
  return from_fbits(sg | ibf(r));
}

// binary64 roundings to an integer on the integer pipe.  b: the bits of x.
// trunc clears the fraction bits; rint and round add half an integer unit
// (less one ulp plus the quotient's low bit for ties to even) to the
// significand and shift; the integer q <= 2^53 is written back exactly.
__device__ __forceinline__ uint64_t trunc_b64(uint64_t b) {
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e >= 52) return b;                                    // integers, infinities, NaNs
  if (e < 0) return b & SIGN64;
  return b & ~(FRAC64 >> e);
}
__device__ __forceinline__ uint64_t from_uint64(uint64_t q) {   // q <= 2^53, exact
  if (q == 0) return 0;
  int p = 63 - __clzll((long long)q);
  return ((uint64_t)(p + 1023) << 52) | ((q << (52 - p)) & FRAC64);
}
template <bool EVEN>
__device__ __forceinline__ uint64_t round_b64(uint64_t b) {
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  uint64_t sg = b & SIGN64;
  if (e >= 52) return b;
  if (e < -1) return sg;                                    // |x| < 1/2
  int s = 52 - e;                                           // 1 .. 53
  uint64_t M = (b & FRAC64) | (1ull << 52), half = 1ull << (s - 1);
  uint64_t add = EVEN ? half - 1 + ((M >> s) & 1) : half;
  return sg | from_uint64((M + add) >> s);
}
// an int32 as a double, exactly, on the integer pipe
__device__ __forceinline__ double from_int32(int v) {
  uint64_t a = (uint64_t)(v < 0 ? -(long long)v : v);
  return from_bits(((uint64_t)(v < 0) << 63) | from_uint64(a));
}

// ---------------- functors: one per function, both formats ----------------
struct Fabs {
  __device__ double operator()(double x) const { return canon_i(from_bits(ib(x) & ABS64)); }
  __device__ float operator()(float x) const { return canonf_i(from_fbits(ibf(x) & ABS32)); }
};
struct Copysign {
  __device__ double operator()(double x, double y) const {
    return canon_i(from_bits((ib(x) & ABS64) | (ib(y) & SIGN64)));
  }
  __device__ float operator()(float x, float y) const {
    return canonf_i(from_fbits((ibf(x) & ABS32) | (ibf(y) & SIGN32)));
  }
};
struct Trunc {
  __device__ double operator()(double x) const { return canon_i(from_bits(trunc_b64(ib(x)))); }
  __device__ float operator()(float x) const { return canonf_i(truncf(x)); }
};
// floor / ceil: trunc on the bits, one step only where the fraction was not
// zero and the sign points that way (|t| < 2^52: exact)
struct Floor {
  __device__ double operator()(double x) const {
    uint64_t b = ib(x), t = trunc_b64(b);
    double r = (t != b && (b >> 63)) ? __dsub_rn(from_bits(t), 1.0) : from_bits(t);
    return canon_i(r);
  }
  __device__ float operator()(float x) const { return canonf_i(floorf(x)); }
};
struct Ceil {
  __device__ double operator()(double x) const {
    uint64_t b = ib(x), t = trunc_b64(b);
    double r = (t != b && !(b >> 63)) ? __dadd_rn(from_bits(t), 1.0) : from_bits(t);
    return canon_i(r);
  }
  __device__ float operator()(float x) const { return canonf_i(ceilf(x)); }
};
struct Rint {
  __device__ double operator()(double x) const { return canon_i(from_bits(round_b64<true>(ib(x)))); }
  __device__ float operator()(float x) const { return canonf_i(rintf(x)); }
};
// ties away from zero.  binary32: t = trunc(x), x - t exact, one step away
// from zero when |x - t| >= 1/2 (only for |x| < 2^23, where t +- 1 is exact)
struct Round {
  __device__ double operator()(double x) const { return canon_i(from_bits(round_b64<false>(ib(x)))); }
  __device__ float operator()(float x) const {
    float t = truncf(x), d = __fsub_rn(x, t);
    bool up = (ibf(d) & ABS32) >= 0x3F000000u && (ibf(d) & ABS32) <= EXP32;
    return canonf_i(up ? __fadd_rn(t, from_fbits((ibf(x) & SIGN32) | 0x3F800000u)) : t);
  }
};
struct Logb {
  __device__ double operator()(double x) const {
    uint64_t ab = ib(x) & ABS64;
    if (ab == 0) return from_bits(SIGN64 | EXP64);
    if (ab >= EXP64) return ab == EXP64 ? from_bits(EXP64) : from_bits(QNAN64);
    return from_int32(expo64(ab));
  }
  __device__ float operator()(float x) const {
    uint32_t ab = ibf(x) & ABS32;
    if (ab == 0) return from_fbits(SIGN32 | EXP32);
    if (ab >= EXP32) return ab == EXP32 ? from_fbits(EXP32) : from_fbits(QNAN32);
    return (float)expo32(ab);
  }
};
struct Ilogb {
  __device__ int32_t operator()(double x) const {
    uint64_t ab = ib(x) & ABS64;
    return ab == 0 ? INT_MIN : (ab >= EXP64 ? INT_MAX : expo64(ab));
  }
  __device__ int32_t operator()(float x) const {
    uint32_t ab = ibf(x) & ABS32;
    return ab == 0 ? INT_MIN : (ab >= EXP32 ? INT_MAX : expo32(ab));
  }
};
struct Ldexp {
  __device__ double operator()(double x, int32_t n) const { return ldexp64(x, n); }
  __device__ float operator()(float x, int32_t n) const { return ldexp32(x, n); }
};
struct Frexp {
  __device__ double operator()(double x, int32_t &k) const {
    uint64_t b = ib(x), ab = b & ABS64;
    k = 0;
    if (ab == 0 || ab >= EXP64) return canon_i(x);
    k = expo64(ab) + 1;
    return from_bits((b & SIGN64) | (mant64(ab) - (1ull << 52)));   // m / 2 in [1/2, 1)
  }
  __device__ float operator()(float x, int32_t &k) const {
    uint32_t b = ibf(x), ab = b & ABS32;
    k = 0;
    if (ab == 0 || ab >= EXP32) return canonf_i(x);
    k = expo32(ab) + 1;
    return from_fbits((b & SIGN32) | (mant32(ab) - (1u << 23)));
  }
};
// modf: fractional part (sign of x, +-0 for integers and infinities) and
// integral part
struct Modf {
  __device__ void operator()(double x, double &fr, double &ip) const {
    uint64_t b = ib(x);
    double t = from_bits(trunc_b64(b));
    double d = (b & ABS64) == EXP64 ? 0.0 : __dsub_rn(x, t);
    fr = from_bits((ib(d) & ABS64) | (b & SIGN64));
    ip = t;
    if ((b & ABS64) > EXP64) fr = ip = from_bits(QNAN64);
  }
  __device__ void dual(float x, float &fr, float &ip) const {
    uint32_t b = ibf(x);
    float t = truncf(x);
    float d = (b & ABS32) == EXP32 ? 0.0f : __fsub_rn(x, t);
    fr = canonf_i(from_fbits((ibf(d) & ABS32) | (b & SIGN32)));
    ip = canonf_i(t);
    if ((b & ABS32) > EXP32) fr = from_fbits(QNAN32);
  }
};
__device__ __forceinline__ long long okey_i(double d) {
  long long b = (long long)ib(d);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ int okey32(float f) {
  int b = (int)ibf(f);
  return b ^ ((b >> 31) & 0x7FFFFFFF);
}
struct Fmax {
  __device__ double operator()(double x, double y) const {
    if (is_nan_b(ib(x))) return canon_i(y);
    if (is_nan_b(ib(y))) return x;
    return okey_i(x) >= okey_i(y) ? x : y;                 // -0 orders below +0
  }
  __device__ float operator()(float x, float y) const {
    if ((ibf(x) & ABS32) > EXP32) return canonf_i(y);
    if ((ibf(y) & ABS32) > EXP32) return x;
    return okey32(x) >= okey32(y) ? x : y;
  }
};
struct Fmin {
  __device__ double operator()(double x, double y) const {
    if (is_nan_b(ib(x))) return canon_i(y);
    if (is_nan_b(ib(y))) return x;
    return okey_i(x) <= okey_i(y) ? x : y;
  }
  __device__ float operator()(float x, float y) const {
    if ((ibf(x) & ABS32) > EXP32) return canonf_i(y);
    if ((ibf(y) & ABS32) > EXP32) return x;
    return okey32(x) <= okey32(y) ? x : y;
  }
};
// x > y ? x - y : +0 (for x = +0, y = -0 both branches give +0)
struct Fdim {
  __device__ double operator()(double x, double y) const {
    if (is_nan_b(ib(x)) || is_nan_b(ib(y))) return from_bits(QNAN64);
    return okey_i(x) > okey_i(y) ? __dsub_rn(x, y) : 0.0;
  }
  __device__ float operator()(float x, float y) const {
    if ((ibf(x) & ABS32) > EXP32 || (ibf(y) & ABS32) > EXP32) return from_fbits(QNAN32);
    return okey32(x) > okey32(y) ? __fsub_rn(x, y) : 0.0f;
  }
};
struct Nextafter {
  __device__ double operator()(double x, double y) const {
    uint64_t bx = ib(x), by = ib(y);
    if (is_nan_b(bx) || is_nan_b(by)) return from_bits(QNAN64);
    if (bx == by || ((bx | by) & ABS64) == 0) return y;
    if ((bx & ABS64) == 0) return from_bits((by & SIGN64) | 1);
    bool away = (okey_i(y) > okey_i(x)) == !(bx >> 63);     // the magnitude grows
    return from_bits(away ? bx + 1 : bx - 1);
  }
  __device__ float operator()(float x, float y) const {
    uint32_t bx = ibf(x), by = ibf(y);
    if ((bx & ABS32) > EXP32 || (by & ABS32) > EXP32) return from_fbits(QNAN32);
    if (bx == by || ((bx | by) & ABS32) == 0) return y;
    if ((bx & ABS32) == 0) return from_fbits((by & SIGN32) | 1);
    bool away = (okey32(y) > okey32(x)) == !(bx >> 31);
    return from_fbits(away ? bx + 1 : bx - 1);
  }
};
struct Sqrt {
  __device__ double operator()(double x) const { return canon_i(__dsqrt_rn(x)); }
  __device__ float operator()(float x) const { return canonf_i(__fsqrt_rn(x)); }
};

// ---------------- hypot ----------------
template <bool U05>
struct Hypot {
  __device__ double operator()(double x, double y) const {
    uint64_t ax = ib(x) & ABS64, ay = ib(y) & ABS64;
    if (ax == EXP64 || ay == EXP64) return from_bits(EXP64);   // an infinity wins over a NaN
    if (ax > EXP64 || ay > EXP64) return from_bits(QNAN64);
    uint64_t ab = ax > ay ? ax : ay, bb = ax > ay ? ay : ax;
    if (bb == 0) return from_bits(ab);
    int e = expo64(ab);
    double as = from_bits(mant64(ab)), b = from_bits(bb), bs;
    if (e >= -1023) {
      bs = dmul(b, pow2_64(-e));                          // one rounding at most
    } else {
      bs = dmul(dmul(b, 0x1p64), pow2_64(-e - 64));   // the first product is exact
    }
    double r;
    if (U05) {
      d2 q = sqrt_d2(add_d2d2_fast(mul_dd(as, as), mul_dd(bs, bs)));
      r = __dadd_rn(q.x, q.y);
    } else {
      r = __dsqrt_rn(__fma_rn(as, as, dmul(bs, bs)));
    }
    return dmul(r, pow2_64(e));                           // one rounding at most
  }
  __device__ float operator()(float x, float y) const {
    uint32_t ax = ibf(x) & ABS32, ay = ibf(y) & ABS32;
    if (ax == EXP32 || ay == EXP32) return from_fbits(EXP32);
    if (ax > EXP32 || ay > EXP32) return from_fbits(QNAN32);
    uint32_t ab = ax > ay ? ax : ay, bb = ax > ay ? ay : ax;
    if (bb == 0) return from_fbits(ab);
    int e = expo32(ab);
    float as = from_fbits(mant32(ab)), b = from_fbits(bb), bs;
    if (e >= -127) {
      bs = __fmul_rn(b, pow2_32(-e));
    } else {
      bs = __fmul_rn(__fmul_rn(b, 0x1p32f), pow2_32(-e - 32));
    }
    float r;
    if (U05) {
      f2 q = sqrt_f2(add_f2f2_fast(mul_ff(as, as), mul_ff(bs, bs)));
      r = __fadd_rn(q.x, q.y);
    } else {
      r = __fsqrt_rn(__fmaf_rn(as, as, __fmul_rn(bs, bs)));
    }
    return __fmul_rn(r, pow2_32(e));
  }
};

// ---------------- sinpi, cospi ----------------
// sin(pi s) = s P(t), cos(pi s) = 1 + t P(t), P = k0 + t (k1 + t (k2 + t p(t)))
// over t = s^2 in [0, 1/16]; k0, k1 DD (FF) pairs, p plain (design constants
// of the minimax fits: sine then cosine)
__device__ constexpr double SK0H = 0x1.921fb54442d18p+1, SK0L = 0x1.1a5ee6df61731p-53;
__device__ constexpr double SK1H = -0x1.4abbce625be53p+2, SK1L = 0x1.1317e21cffea3p-52;
__device__ constexpr double SK2 = 0x1.466bc6775aad9p+1;
__device__ constexpr double SP[5] = {-0x1.32d2cce62ac1bp-1, 0x1.50783485cd9dep-4, -0x1.e3074b54cb043p-8,
                                     0x1.e8eed5bfbbb87p-12, -0x1.6c5d06da75ea5p-16};
__device__ constexpr double CK0H = -0x1.3bd3cc9be45dep+2, CK0L = -0x1.692b254f96cb6p-52;
__device__ constexpr double CK1 = 0x1.03c1f081b5ac4p+2;
__device__ constexpr double CK2 = -0x1.55d3c7e3cc16cp+0;
__device__ constexpr double CP[5] = {0x1.e1f5068965fb7p-3, -0x1.a6d1f30fc0185p-6, 0x1.f9d42dc364f31p-10,
                                     -0x1.b7598d34a382dp-14, 0x1.41f35eddaaed2p-18};
__device__ constexpr float SK0Hf = 0x1.921fb6p+1f, SK0Lf = -0x1.777a6p-24f;
__device__ constexpr float SK1Hf = -0x1.4abbcep+2f, SK1Lf = -0x1.895f1ep-24f;
__device__ constexpr float SK2f = 0x1.466bc6p+1f;
__device__ constexpr float SPf[3] = {-0x1.32d242p-1f, 0x1.5011b4p-4f, -0x1.b11644p-8f};
__device__ constexpr float CK0Hf = -0x1.3bd3ccp+2f, CK0Lf = -0x1.37c6bap-23f;
__device__ constexpr float CK1f = 0x1.03c1f0p+2f;
__device__ constexpr float CK2f = -0x1.55d302p+0f;
__device__ constexpr float CPf[3] = {0x1.e1474ap-3f, -0x1.76f7fcp-6f, 0.0f};

template <bool COS, bool U05>
struct Sincospi {
  __device__ double operator()(double x) const {
    uint64_t b = ib(x), ab = b & ABS64;
    if (ab >= EXP64) return from_bits(QNAN64);
    double s = 0.0;
    int o = 0;
    if (ab < 0x4340000000000000ull) {                          // |x| < 2^53: x = q/2 + s exactly
      double q = drint(__dadd_rn(x, x));
      o = low2_of_int(q);
      s = __fma_rn(-0.5, q, x);
    }
    o = (o + COS) & 3;
    bool c = o & 1;                                            // the cosine polynomial of s
    double pc[5];
#pragma unroll
    for (int i = 0; i < 5; i++) pc[i] = c ? CP[i] : SP[i];
    double k2 = c ? CK2 : SK2;
    double v;
    if (U05) {
      bool tiny = !c && (ib(s) & ABS64) < 0x20B0000000000000ull;   // |s| < 2^-500
      if (tiny) s = dmul(s, 0x1p200);
      d2 t = mul_dd(s, s);
      double p = poly(t.x, pc);
      d2 P = add_dd(k2, dmul(t.x, p));
      P = add_d2d2(c ? D2(CK1, 0.0) : D2(SK1H, SK1L), mul_d2d2(t, P));
      P = add_d2d2(c ? D2(CK0H, CK0L) : D2(SK0H, SK0L), mul_d2d2(t, P));
      d2 r = c ? add_d_d2(1.0, mul_d2d2(t, P)) : mul_d2_d(P, s);
      v = __dadd_rn(r.x, r.y);
      if (tiny) v = dmul(v, 0x1p-200);
    } else {
      double t = dmul(s, s);
      double p = poly(t, pc);
      double P = __fma_rn(t, __fma_rn(t, __fma_rn(t, p, k2), c ? CK1 : SK1H), c ? CK0H : SK0H);
      v = c ? __fma_rn(t, P, 1.0) : dmul(s, P);
    }
    v = neg_if(v, o & 2);
    // zero results: sinpi(n) = +-0 with the sign of n, cospi(n + 1/2) = +0
    if ((ib(v) & ABS64) == 0) v = COS ? 0.0 : from_bits(b & SIGN64);
    return v;
  }
  __device__ float operator()(float x) const {
    uint32_t b = ibf(x), ab = b & ABS32;
    if (ab >= EXP32) return from_fbits(QNAN32);
    float s = 0.0f;
    int o = 0;
    if (ab < 0x4B800000u) {                                    // |x| < 2^24
      float q = rintf(__fadd_rn(x, x));
      o = low2_of_intf(q);
      s = __fmaf_rn(-0.5f, q, x);
    }
    o = (o + COS) & 3;
    bool c = o & 1;
    float pc[3];
#pragma unroll
    for (int i = 0; i < 3; i++) pc[i] = c ? CPf[i] : SPf[i];
    float k2 = c ? CK2f : SK2f;
    float v;
    if (U05) {
      bool tiny = !c && (ibf(s) & ABS32) < 0x0D800000u;     // |s| < 2^-100
      if (tiny) s = __fmul_rn(s, 0x1p80f);
      f2 t = mul_ff(s, s);
      float p = polyf(t.x, pc);
      f2 P = add_ff(k2, __fmul_rn(t.x, p));
      P = add_f2f2(c ? F2(CK1f, 0.0f) : F2(SK1Hf, SK1Lf), mul_f2f2(t, P));
      P = add_f2f2(c ? F2(CK0Hf, CK0Lf) : F2(SK0Hf, SK0Lf), mul_f2f2(t, P));
      f2 r = c ? add_f_f2(1.0f, mul_f2f2(t, P)) : mul_f2_f(P, s);
      v = __fadd_rn(r.x, r.y);
      if (tiny) v = __fmul_rn(v, 0x1p-80f);
    } else {
      float t = __fmul_rn(s, s);
      float p = polyf(t, pc);
      float P = __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, p, k2), c ? CK1f : SK1Hf), c ? CK0Hf : SK0Hf);
      v = c ? __fmaf_rn(t, P, 1.0f) : __fmul_rn(s, P);
    }
    v = negf_if(v, o & 2);
    if ((ibf(v) & ABS32) == 0) v = COS ? 0.0f : from_fbits(b & SIGN32);
    return v;
  }
};

using SinpiU05 = Sincospi<false, true>;
using SinpiU35 = Sincospi<false, false>;
using CospiU05 = Sincospi<true, true>;
using CospiU35 = Sincospi<true, false>;
using HypotU05 = Hypot<true>;
using HypotU35 = Hypot<false>;

// ---------------- kernels with an int32 operand or result ----------------
// 16-byte accesses for the floating-point side: pairs of doubles with int2,
// quadruples of floats with int4.
template <class T> struct Vec;
template <> struct Vec<double> { using TV = double2; using IV = int2; static constexpr int N = 2; };
template <> struct Vec<float> { using TV = float4; using IV = int4; static constexpr int N = 4; };

// ilogb: out[i] = F(x[i])
template <class T, class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_toint(const T *x, int32_t *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    constexpr int N = Vec<T>::N;
    using TV = typename Vec<T>::TV;
    using IV = typename Vec<T>::IV;
    size_t nv = n / N;
    for (size_t i = tid; i < nv; i += stride) {
      TV v = __ldcs(reinterpret_cast<const TV *>(x) + i);
      const T *pv = reinterpret_cast<const T *>(&v);
      IV r;
      int32_t *pr = reinterpret_cast<int32_t *>(&r);
#pragma unroll
      for (int j = 0; j < N; j++) pr[j] = f(pv[j]);
      __stcs(reinterpret_cast<IV *>(out) + i, r);
    }
    size_t rem = n - nv * N;
    if (tid < rem) out[nv * N + tid] = f(x[nv * N + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i]);
  }
}
// ldexp: out[i] = F(x[i], e[i])
template <class T, class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_withint(const T *x, const int32_t *e, T *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    constexpr int N = Vec<T>::N;
    using TV = typename Vec<T>::TV;
    using IV = typename Vec<T>::IV;
    size_t nv = n / N;
    for (size_t i = tid; i < nv; i += stride) {
      TV v = __ldcs(reinterpret_cast<const TV *>(x) + i);
      IV k = __ldcs(reinterpret_cast<const IV *>(e) + i);
      const T *pv = reinterpret_cast<const T *>(&v);
      const int32_t *pk = reinterpret_cast<const int32_t *>(&k);
      TV r;
      T *pr = reinterpret_cast<T *>(&r);
#pragma unroll
      for (int j = 0; j < N; j++) pr[j] = f(pv[j], pk[j]);
      __stcs(reinterpret_cast<TV *>(out) + i, r);
    }
    size_t rem = n - nv * N;
    if (tid < rem) out[nv * N + tid] = f(x[nv * N + tid], e[nv * N + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i], e[i]);
  }
}
// frexp: m[i] = F(x[i], k[i])
template <class T, class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_splitint(const T *x, T *m, int32_t *e, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    constexpr int N = Vec<T>::N;
    using TV = typename Vec<T>::TV;
    using IV = typename Vec<T>::IV;
    size_t nv = n / N;
    for (size_t i = tid; i < nv; i += stride) {
      TV v = __ldcs(reinterpret_cast<const TV *>(x) + i);
      const T *pv = reinterpret_cast<const T *>(&v);
      TV r;
      IV k;
      T *pr = reinterpret_cast<T *>(&r);
      int32_t *pk = reinterpret_cast<int32_t *>(&k);
#pragma unroll
      for (int j = 0; j < N; j++) pr[j] = f(pv[j], pk[j]);
      __stcs(reinterpret_cast<TV *>(m) + i, r);
      __stcs(reinterpret_cast<IV *>(e) + i, k);
    }
    size_t rem = n - nv * N;
    if (tid < rem) {
      int32_t k;
      m[nv * N + tid] = f(x[nv * N + tid], k);
      e[nv * N + tid] = k;
    }
  } else {
    for (size_t i = tid; i < n; i += stride) {
      int32_t k;
      m[i] = f(x[i], k);
      e[i] = k;
    }
  }
}

template <class T>
inline bool aligned_v(const void *p) { return ((uintptr_t)p & (sizeof(typename Vec<T>::IV) - 1)) == 0; }

template <class T, class F>
sleefcu_status launch_toint(const char *name, const T *x, int32_t *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned_v<T>(out)) {
    auto k = k_toint<T, F, true>;
    k<<<grid_for((const void *)k, (n + Vec<T>::N - 1) / Vec<T>::N), kBlock, 0, st>>>(x, out, n);
  } else {
    auto k = k_toint<T, F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, out, n);
  }
  return check_launch(name);
}
template <class T, class F>
sleefcu_status launch_withint(const char *name, const T *x, const int32_t *e, T *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !e || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, e, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(out) && aligned_v<T>(e)) {
    auto k = k_withint<T, F, true>;
    k<<<grid_for((const void *)k, (n + Vec<T>::N - 1) / Vec<T>::N), kBlock, 0, st>>>(x, e, out, n);
  } else {
    auto k = k_withint<T, F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, e, out, n);
  }
  return check_launch(name);
}
template <class T, class F>
sleefcu_status launch_splitint(const char *name, const T *x, T *m, int32_t *e, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !m || !e) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, m, e)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(m) && aligned_v<T>(e)) {
    auto k = k_splitint<T, F, true>;
    k<<<grid_for((const void *)k, (n + Vec<T>::N - 1) / Vec<T>::N), kBlock, 0, st>>>(x, m, e, n);
  } else {
    auto k = k_splitint<T, F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, m, e, n);
  }
  return check_launch(name);
}

}  // namespace c99
}  // namespace sleefcu

using namespace sleefcu;

#define C99_U64(NAME, F)                                                                      \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n, sleefcu_stream s) { \
    return launch_unary64<c99::F>("sleefcu_" #NAME, x, out, n, s);                           \
  }
#define C99_U32(NAME, F)                                                                      \
  extern "C" sleefcu_status sleefcu_##NAME(const float *x, float *out, size_t n, sleefcu_stream s) { \
    return launch_unary32<c99::F>("sleefcu_" #NAME, x, out, n, s);                           \
  }
#define C99_B64(NAME, F)                                                                      \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, const double *y, double *out, size_t n, \
                                           sleefcu_stream s) {                                \
    return launch_binary64<c99::F>("sleefcu_" #NAME, x, y, out, n, s);                       \
  }
#define C99_B32(NAME, F)                                                                      \
  extern "C" sleefcu_status sleefcu_##NAME(const float *x, const float *y, float *out, size_t n, \
                                           sleefcu_stream s) {                                \
    return launch_binary32<c99::F>("sleefcu_" #NAME, x, y, out, n, s);                       \
  }

C99_U64(fabs_f64, Fabs)
C99_U64(trunc_f64, Trunc)
C99_U64(floor_f64, Floor)
C99_U64(ceil_f64, Ceil)
C99_U64(round_f64, Round)
C99_U64(rint_f64, Rint)
C99_U64(logb_f64, Logb)
C99_U64(sqrt_u05_f64, Sqrt)
C99_U64(sqrt_u35_f64, Sqrt)
C99_U64(sinpi_u05_f64, SinpiU05)
C99_U64(sinpi_u35_f64, SinpiU35)
C99_U64(cospi_u05_f64, CospiU05)
C99_U64(cospi_u35_f64, CospiU35)
C99_B64(copysign_f64, Copysign)
C99_B64(fmax_f64, Fmax)
C99_B64(fmin_f64, Fmin)
C99_B64(fdim_f64, Fdim)
C99_B64(nextafter_f64, Nextafter)
C99_B64(hypot_u05_f64, HypotU05)
C99_B64(hypot_u35_f64, HypotU35)

C99_U32(fabs_f32, Fabs)
C99_U32(trunc_f32, Trunc)
C99_U32(floor_f32, Floor)
C99_U32(ceil_f32, Ceil)
C99_U32(round_f32, Round)
C99_U32(rint_f32, Rint)
C99_U32(logb_f32, Logb)
C99_U32(sqrt_u05_f32, Sqrt)
C99_U32(sqrt_u35_f32, Sqrt)
C99_U32(sinpi_u05_f32, SinpiU05)
C99_U32(sinpi_u35_f32, SinpiU35)
C99_U32(cospi_u05_f32, CospiU05)
C99_U32(cospi_u35_f32, CospiU35)
C99_B32(copysign_f32, Copysign)
C99_B32(fmax_f32, Fmax)
C99_B32(fmin_f32, Fmin)
C99_B32(fdim_f32, Fdim)
C99_B32(nextafter_f32, Nextafter)
C99_B32(hypot_u05_f32, HypotU05)
C99_B32(hypot_u35_f32, HypotU35)

extern "C" sleefcu_status sleefcu_modf_f64(const double *x, double *frac, double *ipart, size_t n, sleefcu_stream s) {
  return launch_dual64<c99::Modf>("sleefcu_modf_f64", x, frac, ipart, n, s);
}
extern "C" sleefcu_status sleefcu_modf_f32(const float *x, float *frac, float *ipart, size_t n, sleefcu_stream s) {
  return launch_dual32<c99::Modf>("sleefcu_modf_f32", x, frac, ipart, n, s);
}
extern "C" sleefcu_status sleefcu_ilogb_f64(const double *x, int32_t *out, size_t n, sleefcu_stream s) {
  return c99::launch_toint<double, c99::Ilogb>("sleefcu_ilogb_f64", x, out, n, s);
}
extern "C" sleefcu_status sleefcu_ilogb_f32(const float *x, int32_t *out, size_t n, sleefcu_stream s) {
  return c99::launch_toint<float, c99::Ilogb>("sleefcu_ilogb_f32", x, out, n, s);
}
extern "C" sleefcu_status sleefcu_ldexp_f64(const double *x, const int32_t *e, double *out, size_t n,
                                            sleefcu_stream s) {
  return c99::launch_withint<double, c99::Ldexp>("sleefcu_ldexp_f64", x, e, out, n, s);
}
extern "C" sleefcu_status sleefcu_ldexp_f32(const float *x, const int32_t *e, float *out, size_t n,
                                            sleefcu_stream s) {
  return c99::launch_withint<float, c99::Ldexp>("sleefcu_ldexp_f32", x, e, out, n, s);
}
extern "C" sleefcu_status sleefcu_frexp_f64(const double *x, double *m, int32_t *e, size_t n, sleefcu_stream s) {
  return c99::launch_splitint<double, c99::Frexp>("sleefcu_frexp_f64", x, m, e, n, s);
}
extern "C" sleefcu_status sleefcu_frexp_f32(const float *x, float *m, int32_t *e, size_t n, sleefcu_stream s) {
  return c99::launch_splitint<float, c99::Frexp>("sleefcu_frexp_f32", x, m, e, n, s);
}
