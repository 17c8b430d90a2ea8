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
// 2008 Section 6 prescribes.  NaN results follow the GB300 FP64 pipe bit
// for bit (measured): a NaN operand is returned quieted (bit 51 set, sign
// and payload kept), choosing b, then c, then a for fma and the second
// operand, then the first for add and mul; an invalid operation (inf * 0,
// inf - inf) returns kDefaultNaN; rint and trunc return a NaN argument
// quieted.
// The header compiles as plain C++ as well (host functions), which is how
// the CPU tests pin it against the host processor's hardware fma.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SFP_HD __host__ __device__ __forceinline__
#define SFP_COLD static __host__ __device__ __noinline__   // rare general paths: out of line
#else
#define SFP_HD static inline
#define SFP_COLD static
#endif

namespace sleefcu {
namespace soft {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kExpMask = 0x7FF0000000000000ull;
constexpr uint64_t kManMask = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHidden = 0x0010000000000000ull;
constexpr uint64_t kInf = 0x7FF0000000000000ull;
constexpr uint64_t kQuiet = 0x0008000000000000ull;
constexpr uint64_t kDefaultNaN = 0xFFF8000000000000ull;

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
SFP_COLD uint64_t fma_special(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t aa = a & ~kSign, ab = b & ~kSign, ac = c & ~kSign;
  if (ab > kInf) return b | kQuiet;
  if (ac > kInf) return c | kQuiet;
  if (aa > kInf) return a | kQuiet;
  uint64_t sp = (a ^ b) & kSign;
  if (aa == kInf || ab == kInf) {
    if (aa == 0 || ab == 0) return kDefaultNaN;           // inf * 0
    if (ac == kInf && (c & kSign) != sp) return kDefaultNaN;   // inf - inf
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
  bool zc = (ec | mc) == 0;
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

// ---- add and mul on their own: a 64-bit datapath, far cheaper than fma ----

// x >> s (0 <= s) with the shifted-out bits ORed into bit 0
SFP_HD uint64_t shr_jam64(uint64_t x, int s) {
  if (s >= 64) return (uint64_t)(x != 0);
  return s ? (x >> s) | (uint64_t)((x << (64 - s)) != 0) : x;
}

// Round-to-nearest-even packing of (sign) m 2^(e - 1085) with m < 2^63 (the
// 53-bit significand in bits 62..10 once normalized, 10 guard bits):
// normalizes m (m != 0), rounds, handles subnormal results and overflow.
SFP_HD uint64_t round_pack64(uint64_t sign, uint64_t m, int e) {
  int lz = clz64(m) - 1;                 // leading bit to bit 62
  m <<= lz;
  e -= lz;                               // value m 2^(e - 1085), m in [2^62, 2^63)
  if (e >= 0x7FF) return sign | kInf;
  if (e <= 0) {                          // subnormal: round at 2^-1074
    m = shr_jam64(m, 1 - e);
    e = 1;
  }
  uint64_t r = m & 0x3FF, q = m >> 10;
  q += (uint64_t)(r > 0x200 || (r == 0x200 && (q & 1)));
  return sign | ((((uint64_t)(e - 1)) << 52) + q);
}

// a + b, every case
SFP_COLD uint64_t add_any(uint64_t a, uint64_t b) {
  uint64_t aa = a & ~kSign, ab = b & ~kSign;
  if (aa >= kInf || ab >= kInf) {                        // NaN or infinity
    if (ab > kInf) return b | kQuiet;
    if (aa > kInf) return a | kQuiet;
    if (aa == kInf && ab == kInf && a != b) return kDefaultNaN;
    return aa == kInf ? a : b;
  }
  if (aa < ab) { uint64_t t = a; a = b; b = t; t = aa; aa = ab; ab = t; }   // |a| >= |b|
  if (ab == 0) return aa == 0 ? (a & b) : a;             // +0 unless both are -0
  int ea = (int)(aa >> 52), eb = (int)(ab >> 52);
  uint64_t ma = (aa & kManMask) | (ea ? kHidden : 0), mb = (ab & kManMask) | (eb ? kHidden : 0);
  ea += !ea;                                             // subnormal: exponent 1, no hidden bit
  eb += !eb;
  ma <<= 10;
  mb = shr_jam64(mb << 10, ea - eb);
  uint64_t m;
  if ((a ^ b) & kSign) {
    m = ma - mb;                                         // >= 0 since |a| >= |b|
    if (m == 0) return 0;                                // exact cancellation: +0
  } else {
    m = ma + mb;                                         // < 2^64
    if (m >> 63) { m = (m >> 1) | (m & 1); ea++; }
  }
  return round_pack64(a & kSign, m, ea);
}

// a b, every case
SFP_COLD uint64_t mul_any(uint64_t a, uint64_t b) {
  uint64_t aa = a & ~kSign, ab = b & ~kSign, sign = (a ^ b) & kSign;
  if (aa >= kInf || ab >= kInf) {
    if (ab > kInf) return b | kQuiet;
    if (aa > kInf) return a | kQuiet;
    if (aa == 0 || ab == 0) return kDefaultNaN;           // inf * 0
    return sign | kInf;
  }
  if (aa == 0 || ab == 0) return sign;
  int ea = (int)(aa >> 52), eb = (int)(ab >> 52);
  uint64_t ma = aa & kManMask, mb = ab & kManMask;
  if (ea) ma |= kHidden; else { int s = clz64(ma) - 11; ma <<= s; ea = 1 - s; }
  if (eb) mb |= kHidden; else { int s = clz64(mb) - 11; mb <<= s; eb = 1 - s; }
  // (ma 2^10)(mb 2^11) in [2^125, 2^127): its high word in [2^61, 2^63), the
  // low word folded into bit 0
  uint64_t xa = ma << 10, xb = mb << 11;
  uint64_t hi = mulhi64(xa, xb), lo = xa * xb;
  uint64_t m = hi | (uint64_t)(lo != 0);
  // a b = (xa xb) 2^(ea + eb - 2171) = hi 2^(ea + eb - 2107) = m 2^(e - 1085), e = ea + eb - 1022
  return round_pack64(sign, m, ea + eb - 1022);
}

// ---- the common case on 32-bit words, the rest through add_any / mul_any ----

// a b: normal operands with a normal result take the short path (the product
// of the 53-bit significands from four 32 x 32 -> 64-bit multiply-adds, the
// top 53 bits rounded with a round bit and a sticky bit); anything else
// (zero, subnormal, infinity, NaN, a subnormal or overflowing result) goes
// through mul_any
SFP_HD uint64_t mul(uint64_t a, uint64_t b) {
  uint32_t ah = (uint32_t)(a >> 32), bh = (uint32_t)(b >> 32);
  int ea = (int)((ah >> 20) & 0x7FF), eb = (int)((bh >> 20) & 0x7FF);
  int be = ea + eb - 1023;                  // biased exponent when the product is below 2^105
  if ((unsigned)(ea - 1) >= 2046u || (unsigned)(eb - 1) >= 2046u || (unsigned)(be - 1) >= 2045u)
    return mul_any(a, b);
  uint32_t Ah = (ah & 0xFFFFFu) | 0x100000u, Al = (uint32_t)a;
  uint32_t Bh = (bh & 0xFFFFFu) | 0x100000u, Bl = (uint32_t)b;
  // P = Ah Bh 2^64 + (Ah Bl + Al Bh) 2^32 + Al Bl = hi 2^64 + mid 2^32 + low, P in [2^104, 2^106)
  uint64_t p0 = (uint64_t)Al * Bl;
  uint64_t m1 = (uint64_t)Ah * Bl + (p0 >> 32);
  uint64_t m2 = (uint64_t)Al * Bh + (uint32_t)m1;
  uint64_t hi = (uint64_t)Ah * Bh + (m1 >> 32) + (m2 >> 32);
  uint32_t mid = (uint32_t)m2, low = (uint32_t)p0;
  int n = (int)(hi >> 41);                  // 1 when P >= 2^105
  uint64_t M = (hi << (12 - n)) | (mid >> (20 + n));          // P >> (52 + n): 53 bits
  uint32_t rbit = (mid >> (19 + n)) & 1u;
  uint32_t sticky = (mid & ((1u << (19 + n)) - 1u)) | low;
  M += rbit & ((uint32_t)(sticky != 0) | (uint32_t)(M & 1));
  return ((a ^ b) & kSign) | ((((uint64_t)(be + n - 1)) << 52) + M);
}

// a + b: normal operands below 2^1022 with a normal result take the short
// path (align by the exponent difference with a sticky bit, one signed
// 64-bit addition, one normalizing shift, round); anything else goes
// through add_any
SFP_HD uint64_t add(uint64_t a, uint64_t b) {
  uint64_t aa = a & ~kSign, ab = b & ~kSign;
  bool sw = aa < ab;
  uint64_t x = sw ? b : a, y = sw ? a : b;                     // |x| >= |y|
  uint64_t ax = sw ? ab : aa, ay = sw ? aa : ab;
  int ex = (int)(ax >> 52), ey = (int)(ay >> 52);
  if (ey == 0 || ex >= 2046) return add_any(a, b);
  uint64_t X = ((ax & kManMask) | kHidden) << 10;              // [2^62, 2^63)
  uint64_t Y = ((ay & kManMask) | kHidden) << 10;
  int d = ex - ey;
  Y = d < 64 ? (d ? (Y >> d) | (uint64_t)((Y << (64 - d)) != 0) : Y) : 1;
  uint64_t S = ((x ^ y) & kSign) ? X - Y : X + Y;
  if (S == 0) return 0;                                        // exact cancellation: +0
  int lz = clz64(S);                                           // 0 only after a carry
  int e = ex + 1 - lz;
  if (e < 1) return add_any(a, b);                             // subnormal result
  S = lz ? S << (lz - 1) : (S >> 1) | (S & 1);                 // leading bit to bit 62
  uint64_t q = S >> 10;
  uint32_t r = (uint32_t)S & 0x3FFu;
  q += (uint64_t)(r > 0x200u || (r == 0x200u && (q & 1)));
  return (x & kSign) | ((((uint64_t)(e - 1)) << 52) + q);
}
SFP_HD uint64_t sub(uint64_t a, uint64_t b) { return add(a, b ^ kSign); }

// rint: round to an integral value, ties to even (the sign of a zero result
// is the sign of the argument)
SFP_HD uint64_t rint(uint64_t x) {
  int e = (int)((x >> 52) & 0x7FF);
  if (e == 0x7FF) return (x & ~kSign) > kInf ? x | kQuiet : x;
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

// trunc: round toward zero to an integral value (NaN quieted, as the pipe does)
SFP_HD uint64_t trunc(uint64_t x) {
  int e = (int)((x >> 52) & 0x7FF);
  if (e == 0x7FF) return (x & ~kSign) > kInf ? x | kQuiet : x;
  if (e >= 1075) return x;                                // already integral
  if (e < 1023) return x & kSign;                         // |x| < 1
  return x & ~((1ull << (1075 - e)) - 1);                 // clear the fraction bits
}

}  // namespace soft
}  // namespace sleefcu
