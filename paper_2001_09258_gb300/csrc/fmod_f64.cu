// FP64 fmod and remainder for sm_103a (exact results; the u35 entry points
// are the same kernels).
//
// Section 5.9 (Algorithm 1) and the Appendix B listing: the remainder is
// found by long division with floating-point digits, r_{k+1} = r_k - q_k d,
// q_k = trunc(nextafter(r_k, 0) * rd) with the fix-ups for 1 < r/d < 3 and
// r == d, r held exactly as a double-double, one reciprocal rd <= 1/d in
// total (recip_lower).  Extension for quotients beyond DBL_MAX (the listing's stated
// limit): each step divides by D = d 2^j, j = max(kmin, ilogb(r) - ilogb(d) -
// 1000), which is the listing itself whenever n/d < 2^1000; a subnormal d
// (kmin = 54) is rescaled by 2^54 once r < d 2^54, as in the listing.
// Elements are grouped in divergence-sorted 2048-element tiles by their expected trip
// count (48 classes, trip_class), so the lanes of a warp leave the loop
// together (the listing's "terminate once every element of the vector is
// done").  Comparisons of the non-negative operands run on the integer pipe.
//
// remainder: fmod(|x|, 2|y|), then |y| subtracted once or twice by comparing
// 2 r with |y| (ties to the even quotient), every subtraction exact.
#include "sleefcu_common.cuh"

namespace sleefcu {
namespace fmod64 {

constexpr int MAXIT = 48;
constexpr uint64_t DMIN = 0x0010000000000000ull;   // bits of DBL_MIN
constexpr uint64_t INF = 0x7FF0000000000000ull;

__device__ __forceinline__ double rdown(double v) {   // nextafter(v, 0) for v > 0 finite
  return from_bits(bits(v) - 1);
}
__device__ __forceinline__ int ilogb_n(uint64_t b) { return (int)((b >> 52) & 0x7FF) - 1023; }
// bits of 2v for the bits b of a non-negative finite v: the exponent field
// plus one for a normal v (beyond the largest finite v this gives a pattern
// above +inf, which compares above every finite value as 2v = +inf does), a
// one-bit shift for a subnormal v (into the normal range where it carries)
__device__ __forceinline__ uint64_t twice_b(uint64_t b) {
  return b < 0x0010000000000000ull ? b << 1 : b + 0x0010000000000000ull;
}
__device__ __forceinline__ double scale_n(double v, int j) {   // v normal, v 2^j normal
  return from_bits(bits(v) + ((uint64_t)(int64_t)j << 52));
}

// The reciprocal the long division multiplies by: at most 1/d and within
// 2^-50 of it (Section 5.9 allows any division that keeps q_k in
// [(r_k/d)/2, r_k/d]): the binary32 reciprocal of d's significand truncated
// to 24 bits (the FP32 pipe), widened exactly, two Newton steps with fma,
// two units in the last place down, and 2^-ilogb(d) applied to the exponent
// field; four FP64-pipe operations instead of a correctly rounded division.
// From d = 2^1021 on (1/d nears the subnormal range) the listing's
// nextafter(1/d, 0).
__device__ __forceinline__ double recip_lower(double d) {
  uint64_t b = bits(d);
  int e = (int)(b >> 52) - 1023;
  if (e >= 1021) return rdown(__ddiv_rn(1.0, d));
  uint64_t man = b & 0x000FFFFFFFFFFFFFull;
  double m = from_bits(0x3FF0000000000000ull | man);
  float rf = __frcp_rn(from_fbits(0x3F800000u | (uint32_t)(man >> 29)));     // in (1/2, 1]
  uint32_t rb = fbits(rf);
  double y = from_bits(((uint64_t)((rb >> 23) + 896) << 52) | ((uint64_t)(rb & 0x7FFFFFu) << 29));
  double t = __fma_rn(-m, y, 1.0);
  y = __fma_rn(y, t, y);
  t = __fma_rn(-m, y, 1.0);
  y = __fma_rn(y, t, y);
  return from_bits(bits(y) - 2 - ((uint64_t)(int64_t)e << 52));
}

// one step of Algorithm 1 (listing's fix-ups), r >= 0
__device__ __forceinline__ d2 step(d2 r, double D, double rD) {
  double q = dtrunc(dmul(rdown(r.x), rD));
  uint64_t brx = bits(r.x), bD = bits(D);
  bool gt = brx > bD;                                    // r.x > D
  if (bits(dmul(3.0, D)) > brx && gt) q = 2.0;
  if (bits(dmul(2.0, D)) > brx && gt) q = 1.0;
  if (brx == bD) q = ((bits(r.y) >> 63) == 0 || (bits(r.y) & ABS64) == 0) ? 1.0 : 0.0;
  return norm_d2(add_d2d2(r, mul_dd(q, -D)));
}

// |x| mod |y| for finite n >= 0 and finite d > 0; COUNT adds the number of
// long-division steps taken to *steps (the diagnostics entry point)
template <bool COUNT = false>
__device__ __forceinline__ double fmod_abs(double n, double d, int *steps = nullptr) {
  uint64_t bd = bits(d);
  bool sub = bd < DMIN;
  double dmin = sub ? dmul(d, 0x1p54) : d;          // exact
  double rd0 = recip_lower(dmin);
  int edm = ilogb_n(bits(dmin));                           // ilogb(d) + kmin
  d2 r = D2(n, 0.0);
  uint64_t bdmin = bits(dmin);
  for (int it = 0; it < MAXIT && (int64_t)bits(r.x) >= (int64_t)bdmin; it++) {
    int j = ilogb_n(bits(r.x)) - edm - 1000;             // j - kmin
    if (j < 0) j = 0;
    r = step(r, j ? scale_n(dmin, j) : dmin, j ? scale_n(rd0, -j) : rd0);
    if (COUNT) ++*steps;
  }
  // the remainder equal to the divisor reads as 0; the divisor is positive
  // and finite, a value with one bit pattern, so comparing the bits is
  // comparing the values (on the integer pipe instead of the FP64 pipe)
  double ret;
  if (sub) {
    r = D2(dmul(r.x, 0x1p54), dmul(r.y, 0x1p54));
    for (int k = 0; k < 4 && (int64_t)bits(r.x) >= (int64_t)bdmin; k++) {
      r = step(r, dmin, rd0);
      if (COUNT) ++*steps;
    }
    ret = dmul(r.x, 0x1p-54);
    if (bits(__dadd_rn(r.x, r.y)) == bdmin) ret = 0.0;
  } else {
    ret = r.x;
    if (bits(__dadd_rn(r.x, r.y)) == bd) ret = 0.0;
  }
  return ret;
}

// expected trip count of n mod d (bits of n >= 0 and of the divisor d > 0;
// for the tile sort only, the results do not depend on it): none when
// n < d or the operands are not a division; otherwise 1 + floor(2 (ilogb n
// - ilogb d) / 101).  Each step of the loop removes about 50.5 bits of the
// exponent difference (53 bits of quotient less what the truncated quotient
// of a reciprocal at most 1/d and nextafter(r, 0) gives up), and n >= d
// with equal exponents takes one step: on the full-set workload this
// estimate equals the oracle's step count for 99 % of the elements, against
// 85 % for ceil((ilogb n - ilogb d) / 52), which put equal-exponent
// operands (a quarter of the array, half of them needing a step) with the
// elements that need none.
constexpr int kTripClasses = 48;
__device__ __forceinline__ int trip_class_b(uint64_t an, uint64_t ad) {
  if (an >= INF || ad == 0 || ad >= INF || an < ad) return 0;
  int t = 1 + 2 * (ilogb_n(an) - ilogb_n(ad)) / 101;
  return t > kTripClasses - 1 ? kTripClasses - 1 : t;
}
__device__ __forceinline__ int trip_class(double x, double y) {
  return trip_class_b(bits(x) & ABS64, bits(y) & ABS64);
}
// remainder divides by 2|y| (no step when y is zero or 2|y| overflows)
__device__ __forceinline__ int trip_class_rem(double x, double y) {
  uint64_t ad = bits(y) & ABS64;
  if (ad == 0 || ad > 0x7FDFFFFFFFFFFFFFull) return 0;
  return trip_class_b(bits(x) & ABS64, ad + 0x0010000000000000ull);
}

struct FmodF {
  static constexpr int NCLS = kTripClasses;
  // 2048-element tiles: the long-division tail spreads over some twenty trip
  // classes, and a larger tile puts more lanes of one class in a warp
  // (measured on the full-FP64-set mix: 12.3 -> 14.0 Gelem/s against 1024)
  static constexpr int SORT_EPT = 8;
  __device__ static int cls(double x, double y) { return trip_class(x, y); }
  __device__ double operator()(double x, double y) const {
    uint64_t bx = bits(x), by = bits(y);
    uint64_t an = bx & ABS64, ad = by & ABS64;
    bool ok = an < INF && ad != 0 && ad < INF;
    double ret = fmod_abs(ok ? from_bits(an) : 0.0, ok ? from_bits(ad) : 1.0);
    ret = from_bits((bits(ret) & ABS64) | (bx & ~ABS64));          // copysign(ret, x)
    if (an < ad) ret = x;
    if (ad == 0 || an >= INF || ad > INF) ret = from_bits(QNAN64);
    return canon(ret);
  }
};

struct RemainderF {
  static constexpr int NCLS = kTripClasses;
  static constexpr int SORT_EPT = 8;                 // as FmodF (13.8 -> 15.2 Gelem/s)
  __device__ static int cls(double x, double y) { return trip_class_rem(x, y); }
  __device__ double operator()(double x, double y) const {
    uint64_t bx = bits(x), by = bits(y);
    uint64_t an = bx & ABS64, ad = by & ABS64;
    bool ok = an < INF && ad != 0 && ad < INF;
    double nn = ok ? from_bits(an) : 0.0, d = ok ? from_bits(ad) : 1.0;
    const uint64_t bd = bits(d);
    double r2 = nn;
    if (bd <= 0x7FDFFFFFFFFFFFFFull) r2 = fmod_abs(nn, from_bits(twice_b(bd)));   // 2|y| finite
    // 2 r2 > |y| (quotient 1, or 2 when r2 >= 3|y|/2), compared on the bits
    // of the non-negative operands: the same outcome as the FP64 comparison
    // of the exact 2 r2 (an overflowing 2 r2 compares above every finite |y|
    // either way), without FP64-pipe additions or comparisons
    if (twice_b(bits(r2)) > bd) {
      r2 = __dsub_rn(r2, d);
      if (!(bits(r2) >> 63) && twice_b(bits(r2)) >= bd) r2 = __dsub_rn(r2, d);
    }
    double ret = neg_if(r2, (bx >> 63) != 0);
    if (ad == INF && an < INF) ret = x;
    if (ad == 0 || an >= INF || ad > INF) ret = from_bits(QNAN64);
    return canon(ret);
  }
};

// number of long-division steps of |x| mod |y| (0 where fmod is not a
// division: non-finite x, zero or non-finite y)
struct FmodSteps {
  __device__ double operator()(double x, double y) const {
    uint64_t an = bits(x) & ABS64, ad = bits(y) & ABS64;
    bool ok = an < INF && ad != 0 && ad < INF;
    int steps = 0;
    fmod_abs<true>(ok ? from_bits(an) : 0.0, ok ? from_bits(ad) : 1.0, &steps);
    return (double)steps;
  }
};

}  // namespace fmod64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define BIN64(NAME, F)                                                                      \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, const double *y, double *out,   \
                                           size_t n, sleefcu_stream s) {                    \
    return launch_sorted64b<fmod64::F>("sleefcu_" #NAME, x, y, out, n, s);                  \
  }
#define BIN64_MASKED(NAME, F)                                                               \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const double *y,           \
                                                    const uint8_t *mask, double *out, size_t n, \
                                                    sleefcu_stream s) {                         \
    return launch_masked64b<fmod64::F>("sleefcu_" #NAME "_masked", x, y, mask, out, n, s);      \
  }
BIN64(fmod_u10_f64, FmodF)
BIN64(fmod_u35_f64, FmodF)
BIN64(remainder_u10_f64, RemainderF)
BIN64(remainder_u35_f64, RemainderF)
BIN64_MASKED(fmod_u10_f64, FmodF)
BIN64_MASKED(fmod_u35_f64, FmodF)
BIN64_MASKED(remainder_u10_f64, RemainderF)
BIN64_MASKED(remainder_u35_f64, RemainderF)
#undef BIN64
#undef BIN64_MASKED

extern "C" sleefcu_status sleefcu_fmod_steps_f64(const double *x, const double *y, double *out, size_t n,
                                                 sleefcu_stream s) {
  return launch_binary64<fmod64::FmodSteps>("sleefcu_fmod_steps_f64", x, y, out, n, s);
}
#endif  // SLEEFCU_FUNCTORS_ONLY
