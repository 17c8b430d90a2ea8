// Exact IEEE 754 binary64 arithmetic on the integer pipe.
//
// Section 4 of the paper rests on IEEE operations being bit-for-bit
// reproducible: any correct implementation of round-to-nearest-even fma,
// add, mul and round-to-integral returns the same bits.  On GB300 the FP64
// pipe issues two thread operations per clock per SM while the integer pipe
// and the issue slots are mostly idle in the FP64 kernels, so some warps can
// run the same operation sequence in software, on 32/64-bit integers, beside
// warps that use the DFMA pipe, and every result stays identical.
//
// Every function here takes and returns the bit patterns of binary64 values
// (uint64_t) and rounds to nearest, ties to even, with subnormal inputs and
// results (no flush to zero), signed zeros, infinities and NaN as IEEE 754
// 2008 Section 6 prescribes.  A NaN result is the quiet NaN kNaN (the
// pattern the device's FP64 pipe produces, so that even NaN bits agree).
// The header compiles as plain C++ as well (host functions), which is how
// the CPU tests pin it against the host processor's hardware fma.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SFP_HD __host__ __device__ __forceinline__
#else
#define SFP_HD static inline
#endif

namespace sleefcu {
namespace soft {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kExpMask = 0x7FF0000000000000ull;
constexpr uint64_t kManMask = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHidden = 0x0010000000000000ull;
constexpr uint64_t kInf = 0x7FF0000000000000ull;
constexpr uint64_t kNaN = 0x7FFFFFFFFFFFFFFFull;

// ---- primitives with host and device forms ----
SFP_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
SFP_HD int clz64(uint64_t x) {   // 64 for x == 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// 128-bit unsigned value hi:lo
struct u128 { uint64_t hi, lo; };

// x >> s for 0 <= s, with every bit shifted out ORed into bit 0 ("jamming")
SFP_HD u128 shr_jam(u128 x, int s) {
  u128 r;
  if (s == 0) return x;
  if (s < 64) {
    r.lo = (x.lo >> s) | (x.hi << (64 - s)) | (uint64_t)((x.lo << (64 - s)) != 0);
    r.hi = x.hi >> s;
  } else if (s < 128) {
    int t = s - 64;
    uint64_t lost = t ? (x.hi << (64 - t)) | x.lo : x.lo;
    r.lo = (t ? x.hi >> t : x.hi) | (uint64_t)(lost != 0);
    r.hi = 0;
  } else {
    r.lo = (uint64_t)((x.hi | x.lo) != 0);
    r.hi = 0;
  }
  return r;
}
SFP_HD u128 shl(u128 x, int s) {   // 0 <= s < 128
  u128 r;
  if (s == 0) return x;
  if (s < 64) {
    r.hi = (x.hi << s) | (x.lo >> (64 - s));
    r.lo = x.lo << s;
  } else {
    r.hi = x.lo << (s - 64);
    r.lo = 0;
  }
  return r;
}
SFP_HD int clz128(u128 x) { return x.hi ? clz64(x.hi) : 64 + clz64(x.lo); }

// The NaN/infinity cases of fma(a, b, c) (some operand has exponent 0x7FF)
SFP_HD uint64_t fma_special(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t aa = a & ~kSign, ab = b & ~kSign, ac = c & ~kSign;
  if (aa > kInf || ab > kInf || ac > kInf) return kNaN;
  uint64_t sp = (a ^ b) & kSign;
  if (aa == kInf || ab == kInf) {
    if (aa == 0 || ab == 0) return kNaN;                  // inf * 0
    if (ac == kInf && (c & kSign) != sp) return kNaN;     // inf - inf
    return sp | kInf;
  }
  return c;                                               // finite a*b + inf
}

// Round-to-nearest-even packing of the exact value (sign) R * 2^E, R != 0:
// normalizes R, rounds to 53 bits (fewer in the subnormal range), handles
// overflow to infinity.
SFP_HD uint64_t round_pack(uint64_t sign, u128 R, int E) {
  int lz = clz128(R);
  R = shl(R, lz);                        // R in [2^127, 2^128): value = R 2^(E - lz)
  int be = E - lz + 1150;                // biased exponent: value = (R >> 75) 2^(be - 1075)
  if (be >= 0x7FF) return sign | kInf;
  int sh = 75;                           // bits below the 53-bit significand
  if (be <= 0) {                         // subnormal result: round at the fixed 2^-1074
    sh += 1 - be;
    be = 1;
  }
  uint64_t m;
  bool gt, eq;                           // remainder above / exactly at half an ulp
  if (sh < 128) {                        // 75 <= sh < 128: the significand comes from R.hi
    int t = sh - 64;                     // 11 <= t <= 63
    m = R.hi >> t;
    uint64_t rem = R.hi & ((1ull << t) - 1), half = 1ull << (t - 1);
    gt = rem > half || (rem == half && R.lo != 0);
    eq = rem == half && R.lo == 0;
  } else {                               // below the least subnormal: 0 or 2^-1074
    m = 0;
    gt = sh == 128 && (R.hi > kSign || (R.hi == kSign && R.lo != 0));
    eq = sh == 128 && R.hi == kSign && R.lo == 0;
  }
  m += (uint64_t)(gt || (eq && (m & 1)));
  // a carry out of the significand moves into the exponent field (and to
  // infinity from the largest finite value)
  return sign | ((((uint64_t)(be - 1)) << 52) + m);
}

// fma(a, b, c) = RN(a b + c), one rounding
SFP_HD uint64_t fma(uint64_t a, uint64_t b, uint64_t c) {
  int ea = (int)((a >> 52) & 0x7FF), eb = (int)((b >> 52) & 0x7FF), ec = (int)((c >> 52) & 0x7FF);
  if (ea == 0x7FF || eb == 0x7FF || ec == 0x7FF) return fma_special(a, b, c);
  uint64_t sp = (a ^ b) & kSign, sc = c & kSign;
  uint64_t ma = a & kManMask, mb = b & kManMask, mc = c & kManMask;
  bool zc = (ea | mc) == 0;
  if ((ea | ma) == 0 || (eb | mb) == 0) {                 // a b = +-0 exactly
    if (zc) return sp & sc;                               // +0 unless both are -0
    return c;
  }
  // significands in [2^52, 2^53) and exponents: value = m 2^(e - 1075)
  if (ea) ma |= kHidden; else { int s = clz64(ma) - 11; ma <<= s; ea = 1 - s; }
  if (eb) mb |= kHidden; else { int s = clz64(mb) - 11; mb <<= s; eb = 1 - s; }
  // P = (ma 2^11)(mb 2^10) in [2^125, 2^127); a b = P 2^Ep
  uint64_t xa = ma << 11, xb = mb << 10;
  u128 P;
  P.hi = mulhi64(xa, xb);
  P.lo = xa * xb;
  int Ep = ea + eb - 2171;
  if (zc) return round_pack(sp, P, Ep);
  if (ec) mc |= kHidden; else { int s = clz64(mc) - 11; mc <<= s; ec = 1 - s; }
  // C = mc 2^73 in [2^125, 2^126); c = C 2^Ec
  u128 C;
  C.hi = mc << 9;
  C.lo = 0;
  int Ec = ec - 1148;
  // align to the larger exponent; the smaller operand is shifted right with
  // the lost bits jammed into bit 0 (at least 70 bits below the rounding
  // position whenever bits are lost, so the rounding is unaffected)
  int d = Ep - Ec, E;
  if (d >= 0) { C = shr_jam(C, d); E = Ep; }
  else { P = shr_jam(P, -d); E = Ec; }
  u128 R;
  uint64_t sign;
  if (sp == sc) {
    R.lo = P.lo + C.lo;
    R.hi = P.hi + C.hi + (uint64_t)(R.lo < P.lo);
    sign = sp;
  } else {
    R.lo = P.lo - C.lo;
    R.hi = P.hi - C.hi - (uint64_t)(P.lo < C.lo);
    sign = sp;
    if (R.hi & kSign) {                                   // |C| > |P|: negate
      R.lo = ~R.lo + 1;
      R.hi = ~R.hi + (uint64_t)(R.lo == 0);
      sign = sc;
    }
    if ((R.hi | R.lo) == 0) return 0;                     // exact cancellation: +0
  }
  return round_pack(sign, R, E);
}

SFP_HD uint64_t mul(uint64_t a, uint64_t b) { return fma(a, b, kSign); }                    // a b + (-0)
SFP_HD uint64_t add(uint64_t a, uint64_t b) { return fma(a, 0x3FF0000000000000ull, b); }    // a 1 + b
SFP_HD uint64_t sub(uint64_t a, uint64_t b) { return add(a, b ^ kSign); }

// rint: round to an integral value, ties to even (the sign of a zero result
// is the sign of the argument)
SFP_HD uint64_t rint(uint64_t x) {
  int e = (int)((x >> 52) & 0x7FF);
  if (e == 0x7FF) return (x & ~kSign) > kInf ? kNaN : x;
  if (e >= 1075) return x;                                // already integral
  uint64_t s = x & kSign;
  if (e < 1022) return s;                                 // |x| < 1/2
  int sh = 1075 - e;                                      // 1 .. 53
  uint64_t m = (x & kManMask) | kHidden;
  uint64_t q = m >> sh, rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  q += (uint64_t)(rem > half || (rem == half && (q & 1)));
  if (q == 0) return s;
  // q 2^sh has the exponent of x, or one more after a carry to 2^53
  return s | ((((uint64_t)(e - 1)) << 52) + (q << sh));
}

}  // namespace soft
}  // namespace sleefcu
