// FP64 asin, acos, atan, atan2 (u10 and u35) for sm_103a.
//
// asin/acos (Section 5.3): |x| <= 0.5 directly, otherwise through
//   asin x = pi/2 - 2 asin(sqrt((1-x)/2)) (acos x = 2 asin(...), and
//   pi - 2 asin(...) for x < -0.5); one arcsine polynomial on [0, 0.5].
// atan (Section 5.4): a' = 1/a for |a| >= 1, one polynomial on [0, 1],
//   pi/2 - r in that case.
// atan2: quotient of the smaller by the larger magnitude in DD, the atan
//   core, pi/2 - r and pi - r reconstructions, C99 Annex F pairs last.
// Lanes are grouped by branch in divergence-sorted tiles (the class is the
// branch a lane takes), so each warp runs one branch.
#include "sleefcu_common.cuh"

namespace sleefcu {
namespace invtrig64 {

constexpr double PIO2H = 0x1.921fb54442d18p0, PIO2L = 0x1.1a62633145c07p-54;
constexpr double PIH = 0x1.921fb54442d18p1, PIL = 0x1.1a62633145c07p-53;
constexpr double PI4 = 0x1.921fb54442d18p-1, PI34 = 0x1.2d97c7f3321d2p1;
constexpr uint64_t ONE = 0x3FF0000000000000ull, HALF = 0x3FE0000000000000ull;
constexpr uint64_t INF = 0x7FF0000000000000ull, DMAX = 0x7FEFFFFFFFFFFFFFull;

static __constant__ double kAsinU10[13] = {
  0x1.5555555555577p-3, 0x1.333333332e131p-4, 0x1.6db6db7212680p-5, 0x1.f1c71a94f2d61p-6,
  0x1.6e8bdee04467bp-6, 0x1.1c49f05c614d5p-6, 0x1.ca1f8d8013edbp-7, 0x1.75858907d1626p-7,
  0x1.613c905725fb1p-7, 0x1.e5f54ce7fcfd8p-9, 0x1.639c82c0224b6p-6, -0x1.57fd8f93ea512p-6,
  0x1.0b46c1e48a247p-5};
constexpr double AT_C1H = -0x1.555555555554dp-2, AT_C1L = 0x1.f6f1c78b4061fp-57;
static __constant__ double kAtanU10[20] = {
  0x1.9999999998c27p-3, -0x1.2492492456a9cp-3, 0x1.c71c71b628925p-4, -0x1.745d15d02799cp-4,
  0x1.3b139bce356edp-4, -0x1.1110326711fe3p-4, 0x1.e1d487be7157ap-5, -0x1.aeda6036339c0p-5,
  0x1.84b4dcab75621p-5, -0x1.5f276ea2a952dp-5, 0x1.3911a513777bbp-5, -0x1.0cba41b2fdaedp-5,
  0x1.ad1808a727ccep-6, -0x1.31f10ec96d5a7p-6, 0x1.75115934da341p-7, -0x1.73826f657b4aap-8,
  0x1.1e67b2bdce61dp-9, -0x1.3de0d575d18fdp-11, 0x1.c1459ac17e788p-14, -0x1.2e664c7ca4205p-17};
static __constant__ double kAtanU35[19] = {
  -0x1.555555555544cp-2, 0x1.999999998410ep-3, -0x1.2492491fa20b6p-3, 0x1.c71c709e18536p-4,
  -0x1.745d0230ed218p-4, 0x1.3b12b2e80c939p-4, -0x1.11089cfe49ae0p-4, 0x1.e1781718de794p-5,
  -0x1.ad32ba2f14c5ep-5, 0x1.7ee3f6bdf7ae1p-5, -0x1.4f4524eb17978p-5, 0x1.1715e3114eceep-5,
  -0x1.a726c401b7411p-6, 0x1.162c5d3e40d3ep-6, -0x1.2cf7a264b90d9p-7, 0x1.f96d516ef2061p-9,
  -0x1.312abcc54c86dp-10, 0x1.d3bc387104c94p-13, -0x1.53e7168f3586cp-16};

__device__ __forceinline__ double copysign_b(double v, uint64_t sgn_src) {
  return from_bits((bits(v) & ABS64) | (sgn_src & ~ABS64));
}

// sqrt of a non-negative double as DD; the tail is 0 for a zero argument
__device__ __forceinline__ d2 sqrt_dd(double t) {
  double h = __dsqrt_rn(t);
  double r = __fma_rn(-h, h, t);
  double lo = dmul(r, __ddiv_rn(1.0, __dadd_rn(h, h)));
  return D2(h, (bits(h) & ABS64) != 0 ? lo : 0.0);
}

__device__ __forceinline__ d2 asin_core_u10(double ax, bool big) {
  d2 u;
  double t;
  if (!big) {
    u = D2(ax, 0.0);
    t = dmul(ax, ax);
  } else {
    t = dmul(__dsub_rn(1.0, ax), 0.5);
    u = sqrt_dd(t);
  }
  double corr = dmul(dmul(u.x, t), poly(t, kAsinU10));
  return add_d2_d_fast(u, corr);
}
// a square root the compiler cannot hoist out of its branch: inlined, the
// 3.5-ULP asin/acos had both arms if-converted, so every lane paid for the
// square root (ncu: 33 FP64 instructions per element on either path)
static __device__ __noinline__ double sqrt_branch(double t) { return __dsqrt_rn(t); }

__device__ __forceinline__ double asin_core_u35(double ax, bool big) {
  double u, t;
  if (!big) {
    u = ax;
    t = dmul(ax, ax);
  } else {
    t = dmul(__dsub_rn(1.0, ax), 0.5);
    u = sqrt_branch(t);
  }
  return __fma_rn(dmul(u, t), poly(t, kAsinU10), u);
}

#define ASIN_CLASSES                     \
  static constexpr int NCLS = 2;         \
  __device__ static int cls(double x) { return (bits(x) & ABS64) > HALF; }

struct AsinU10 {
  ASIN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    double ax = from_bits(ab);
    bool big = ab > HALF;
    d2 r = asin_core_u10(ax, big);
    if (big) r = add_d2d2_fast(D2(PIO2H, PIO2L), scale_d2(r, -2.0));
    double y = copysign_b(__dadd_rn(r.x, r.y), b);
    if (ab > ONE) y = from_bits(QNAN64);
    return canon(y);
  }
};
struct AcosU10 {
  ASIN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    double ax = from_bits(ab);
    bool big = ab > HALF, neg = (b >> 63) && ab != 0;
    d2 r = asin_core_u10(ax, big), s;
    if (!big) s = add_d2d2_fast(D2(PIO2H, PIO2L), neg ? r : D2(-r.x, -r.y));
    else if (!neg) s = scale_d2(r, 2.0);
    else s = add_d2d2_fast(D2(PIH, PIL), scale_d2(r, -2.0));
    double y = __dadd_rn(s.x, s.y);
    if (ab > ONE) y = from_bits(QNAN64);
    return canon(y);
  }
};
struct AsinU35 {
  ASIN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    bool big = ab > HALF;
    double r = asin_core_u35(from_bits(ab), big);
    if (big) r = __dadd_rn(__fma_rn(-2.0, r, PIO2H), PIO2L);
    double y = copysign_b(r, b);
    if (ab > ONE) y = from_bits(QNAN64);
    return canon(y);
  }
};
struct AcosU35 {
  ASIN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    bool big = ab > HALF, neg = (b >> 63) && ab != 0;
    double r = asin_core_u35(from_bits(ab), big), y;
    if (!big) y = __dadd_rn(__dsub_rn(PIO2H, copysign_b(r, b)), PIO2L);
    else if (!neg) y = dmul(2.0, r);
    else y = __dadd_rn(__fma_rn(-2.0, r, PIH), PIL);
    if (ab > ONE) y = from_bits(QNAN64);
    return canon(y);
  }
};

// atan(s), s in [0, 1] as DD: s + s t (c1 + t P(t))
__device__ __forceinline__ d2 atan_core_u10(d2 s) {
  d2 t = sqr_d2(s);
  double p = poly(t.x, kAtanU10);
  d2 w = add_d2_d_fast(D2(AT_C1H, AT_C1L), dmul(t.x, p));
  w = mul_d2d2(t, w);
  w = mul_d2d2(s, w);
  return add_d2d2_fast(s, w);
}
__device__ __forceinline__ double atan_core_u35(double s) {
  double t = dmul(s, s);
  return __fma_rn(dmul(s, t), poly(t, kAtanU35), s);
}

#define ATAN_CLASSES                     \
  static constexpr int NCLS = 2;         \
  __device__ static int cls(double x) { return (bits(x) & ABS64) >= ONE; }

struct AtanU10 {
  ATAN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    double ax = from_bits(ab);
    bool big = ab >= ONE;
    d2 s = big ? rec_d(ax) : D2(ax, 0.0);
    if (ab == INF) s = D2(0.0, 0.0);
    d2 r = atan_core_u10(s);
    if (big) r = add_d2d2_fast(D2(PIO2H, PIO2L), D2(-r.x, -r.y));
    return canon(copysign_b(__dadd_rn(r.x, r.y), b));
  }
};
struct AtanU35 {
  ATAN_CLASSES
  __device__ double operator()(double x) const {
    uint64_t b = bits(x), ab = b & ABS64;
    double ax = from_bits(ab);
    bool big = ab >= ONE;
    double r = atan_core_u35(big ? __ddiv_rn(1.0, ax) : ax);
    if (big) r = __dsub_rn(PIO2H, r);
    return canon(copysign_b(r, b));
  }
};

// Annex F special pairs of atan2(a, b)
__device__ __forceinline__ bool atan2_special(uint64_t ba, uint64_t bb, double &y) {
  uint64_t aa = ba & ABS64, ab = bb & ABS64;
  if (aa > INF || ab > INF) { y = from_bits(QNAN64); return true; }
  if (ab == INF) {
    bool bpos = (bb >> 63) == 0;
    if (aa == INF) y = copysign_b(bpos ? PI4 : PI34, ba);
    else y = copysign_b(bpos ? 0.0 : PIH, ba);
    return true;
  }
  if (aa == INF) { y = copysign_b(PIO2H, ba); return true; }
  if (aa == 0 && ab == 0) { y = copysign_b((bb >> 63) ? PIH : 0.0, ba); return true; }
  return false;
}

#define ATAN2_CLASSES                            \
  static constexpr int NCLS = 2;                 \
  __device__ static int cls(double a, double b) { return (bits(a) & ABS64) > (bits(b) & ABS64); }

struct Atan2U10 {
  ATAN2_CLASSES
  __device__ double operator()(double a, double b) const {
    uint64_t ba = bits(a), bb = bits(b);
    uint64_t aa = ba & ABS64, ab = bb & ABS64;
    bool swap = aa > ab;
    uint64_t num = swap ? ab : aa, den = swap ? aa : ab;
    if (!((den - 1) < DMAX) || !(num <= den)) { num = 0; den = ONE; }
    double fn = from_bits(num), fd = from_bits(den);
    if (den < 0x0170000000000000ull) { fn = dmul(fn, 0x1p600); fd = dmul(fd, 0x1p600); }
    if (den > 0x7E70000000000000ull) { fn = dmul(fn, 0x1p-600); fd = dmul(fd, 0x1p-600); }
    d2 s = div_d2d2(D2(fn, 0.0), D2(fd, 0.0));
    d2 r = atan_core_u10(s);
    if (swap) r = add_d2d2_fast(D2(PIO2H, PIO2L), D2(-r.x, -r.y));
    bool bneg = (bb >> 63) && ab != 0 && ab <= INF;   // b < 0
    if (bneg) r = add_d2d2_fast(D2(PIH, PIL), D2(-r.x, -r.y));
    double y = copysign_b(__dadd_rn(r.x, r.y), ba);
    atan2_special(ba, bb, y);
    return canon(y);
  }
};
struct Atan2U35 {
  ATAN2_CLASSES
  __device__ double operator()(double a, double b) const {
    uint64_t ba = bits(a), bb = bits(b);
    uint64_t aa = ba & ABS64, ab = bb & ABS64;
    bool swap = aa > ab;
    uint64_t num = swap ? ab : aa, den = swap ? aa : ab;
    if (!((den - 1) < DMAX) || !(num <= den)) { num = 0; den = ONE; }
    double fn = from_bits(num), fd = from_bits(den);
    if (den < 0x0170000000000000ull) { fn = dmul(fn, 0x1p600); fd = dmul(fd, 0x1p600); }
    if (den > 0x7E70000000000000ull) { fn = dmul(fn, 0x1p-600); fd = dmul(fd, 0x1p-600); }
    double r = atan_core_u35(dmul(fn, __ddiv_rn(1.0, fd)));
    if (swap) r = __dsub_rn(PIO2H, r);
    bool bneg = (bb >> 63) && ab != 0 && ab <= INF;
    if (bneg) r = __dsub_rn(PIH, r);
    double y = copysign_b(r, ba);
    atan2_special(ba, bb, y);
    return canon(y);
  }
};

}  // namespace invtrig64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define SORTED64(NAME, F)                                                                   \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_sorted64<invtrig64::F>("sleefcu_" #NAME, x, out, n, s);                   \
  }
#define SORTED64_MASKED(NAME, F)                                                    \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<invtrig64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
SORTED64(asin_u10_f64, AsinU10)
SORTED64_MASKED(asin_u10_f64, AsinU10)
SORTED64(asin_u35_f64, AsinU35)
SORTED64_MASKED(asin_u35_f64, AsinU35)
SORTED64(acos_u10_f64, AcosU10)
SORTED64_MASKED(acos_u10_f64, AcosU10)
SORTED64(acos_u35_f64, AcosU35)
SORTED64_MASKED(acos_u35_f64, AcosU35)
SORTED64(atan_u10_f64, AtanU10)
SORTED64_MASKED(atan_u10_f64, AtanU10)
SORTED64(atan_u35_f64, AtanU35)
SORTED64_MASKED(atan_u35_f64, AtanU35)

extern "C" sleefcu_status sleefcu_atan2_u10_f64(const double *x, const double *y, double *out, size_t n,
                                                sleefcu_stream s) {
  return launch_sorted64b<invtrig64::Atan2U10>("sleefcu_atan2_u10_f64", x, y, out, n, s);
}
extern "C" sleefcu_status sleefcu_atan2_u35_f64(const double *x, const double *y, double *out, size_t n,
                                                sleefcu_stream s) {
  return launch_sorted64b<invtrig64::Atan2U35>("sleefcu_atan2_u35_f64", x, y, out, n, s);
}
extern "C" sleefcu_status sleefcu_atan2_u10_f64_masked(const double *x, const double *y, const uint8_t *mask,
                                                       double *out, size_t n, sleefcu_stream s) {
  return launch_masked64b<invtrig64::Atan2U10>("sleefcu_atan2_u10_f64_masked", x, y, mask, out, n, s);
}
extern "C" sleefcu_status sleefcu_atan2_u35_f64_masked(const double *x, const double *y, const uint8_t *mask,
                                                       double *out, size_t n, sleefcu_stream s) {
  return launch_masked64b<invtrig64::Atan2U35>("sleefcu_atan2_u35_f64_masked", x, y, mask, out, n, s);
}
#undef SORTED64
#undef SORTED64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
