// Structured random operands for the checks of the software binary64
// arithmetic: uniform bit patterns, cancellation, subnormal and overflow
// ranges, few-bit significands (exact ties), specials, additions and
// products.  Shared by the host check (softfp_check.cc) and the device check
// (softfp_gpu.cu); test infrastructure.
#pragma once
#include <stdint.h>
#include <string.h>

#include "../../paper_2001_09258_gb300/csrc/softfp64.cuh"

#if defined(__CUDACC__)
#define GEN_HD __host__ __device__ __forceinline__
#define GEN_M __host__ __device__ __forceinline__
#else
#define GEN_HD static inline
#define GEN_M inline
#endif

namespace S = sleefcu::soft;

GEN_HD uint64_t b_of(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
GEN_HD double d_of(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
GEN_HD bool is_nan(uint64_t u) { return (u & ~S::kSign) > S::kInf; }

// splitmix64
struct Rng {
  uint64_t s;
  GEN_M uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  GEN_M int range(int lo, int hi) { return lo + (int)(next() % (uint64_t)(hi - lo + 1)); }
};

GEN_HD uint64_t special(int i) {
  const uint64_t kSpecials[] = {
    0x0000000000000000ull, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
    0x7FF8000000000000ull, 0xFFF8000000000001ull, 0x7FF0000000000001ull, 0x0000000000000001ull,
    0x8000000000000001ull, 0x000FFFFFFFFFFFFFull, 0x0010000000000000ull, 0x7FEFFFFFFFFFFFFFull,
    0xFFEFFFFFFFFFFFFFull, 0x3FF0000000000000ull, 0xBFF0000000000000ull, 0x3FE0000000000000ull,
    0x0008000000000000ull, 0x7FE0000000000000ull, 0x3CA0000000000000ull, 0x4330000000000000ull};
  return kSpecials[i];
}
constexpr int kNSpecials = 20;

// a finite value with biased exponent e (0: subnormal) and a random significand
GEN_HD uint64_t with_exp(Rng &r, int e, int sig_bits) {
  uint64_t m = r.next() & S::kManMask;
  if (sig_bits < 52) m &= ~((1ull << (52 - sig_bits)) - 1);   // few significant bits: exact ties
  return (r.next() & S::kSign) | ((uint64_t)e << 52) | m;
}

// one random triple in the given mode
GEN_HD void gen(Rng &r, int mode, uint64_t &a, uint64_t &b, uint64_t &c) {
  switch (mode) {
    case 0:                              // uniform bit patterns
      a = r.next(); b = r.next(); c = r.next();
      break;
    case 1: {                            // cancellation: c near -RN(a b)
      a = with_exp(r, r.range(900, 1150), 52); b = with_exp(r, r.range(900, 1150), 52);
      uint64_t p = S::mul(a, b) ^ S::kSign;      // checked on its own in the other modes
      int k = r.range(-4, 4);
      c = (p & S::kExpMask) && (p & S::kExpMask) != S::kExpMask ? p + (uint64_t)(int64_t)k : p;
      break;
    }
    case 2:                              // subnormal and near-underflow products and addends
      a = with_exp(r, r.range(0, 600), r.range(1, 52)); b = with_exp(r, r.range(0, 560), r.range(1, 52));
      c = r.range(0, 3) ? with_exp(r, r.range(0, 60), r.range(1, 52)) : (r.next() & S::kSign);
      break;
    case 3:                              // near overflow
      a = with_exp(r, r.range(1000, 2046), 52); b = with_exp(r, r.range(1000, 1100), 52);
      c = with_exp(r, r.range(2000, 2046), r.range(1, 52));
      break;
    case 4: {                            // few significant bits: exact ties of products and sums
      int ea = r.range(900, 1150), eb = r.range(900, 1150);
      a = with_exp(r, ea, r.range(1, 30)); b = with_exp(r, eb, r.range(1, 30));
      int ec = ea + eb - 1023 + r.range(-60, 60);
      c = ec > 0 && ec < 2047 ? with_exp(r, ec, r.range(1, 52)) : 0;
      break;
    }
    case 5:                              // specials mixed with random finite values
      a = r.range(0, 1) ? special(r.range(0, kNSpecials - 1)) : with_exp(r, r.range(0, 2046), 52);
      b = r.range(0, 1) ? special(r.range(0, kNSpecials - 1)) : with_exp(r, r.range(0, 2046), 52);
      c = r.range(0, 1) ? special(r.range(0, kNSpecials - 1)) : with_exp(r, r.range(0, 2046), 52);
      break;
    case 6: {                            // additions: b a power of two, exponents of a and c close
      int ea = r.range(1, 2046);
      a = with_exp(r, ea, r.range(1, 52));
      b = (r.next() & S::kSign) | ((uint64_t)r.range(1000, 1046) << 52);
      int ec = ea + (int)((b >> 52) & 0x7FF) - 1023 + r.range(-60, 60);
      c = ec > 0 && ec < 2047 ? with_exp(r, ec, r.range(1, 52)) : with_exp(r, r.range(0, 2046), 52);
      break;
    }
    default:                             // products: c = +-0
      a = with_exp(r, r.range(0, 2046), r.range(1, 52)); b = with_exp(r, r.range(0, 2046), r.range(1, 52));
      c = r.next() & S::kSign;
      break;
  }
}

