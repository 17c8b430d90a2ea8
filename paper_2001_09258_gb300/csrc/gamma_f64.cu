// FP64 tgamma and lgamma (u10; the u35 entry points run the same kernels)
// for sm_103a.  The paper lists both in the library without their steps;
// the design, as in the oracle:
//   y >= 8           Stirling: (y - 1/2) log y - y + log(2 pi)/2 + G(1/y^2)/y
//                    with the DD logarithm of pow (Section 5.7)
//   1.75 <= y < 2.5  lgamma(2 + e) = e (c1 + e (c2 + e P(e))), e = y - 2
//   1.25 <= y < 1.75 lgamma(1.5 + u) = c0 + u (c1 + u (c2 + u P(u)))
//   0.5 <= y < 1.25  lgamma(y + 1) - log y with those polynomials
//   otherwise        lgamma(y + n) - log(y (y+1) ... (y+n-1)), y + n in [8, 9)
//   y < 0            log pi - log|sin(pi y)| - lgamma(1 - y), sin(pi y) from
//                    y reduced exactly to [-1/2, 1/2]
// tgamma = sign * exp(L) with L the DD log-gamma.  Lanes are grouped by path
// in sorted tiles (the shift path runs a loop of up to seven DD products).
//
// Multiplications run in software on the integer pipe through one
// out-of-line copy of the exact multiply (SLEEFCU_SOFT_MUL 2 for this
// translation unit), with four resident blocks per SM.  Measured on GB300
// on 2^25 elements of the full-set workload: tgamma 2.09 Gelem/s with the
// FP64 pipe's multiply, 1.45 with the software multiply inlined at its many
// call sites (the paths of eight classes in one kernel), 2.42 out of line;
// lgamma 4.46, 3.74, 5.37.  The results are the same bits in all three.
#ifndef SLEEFCU_FUNCTORS_ONLY
#define SLEEFCU_SOFT_MUL 2
#endif
#include "explog64_core.cuh"

namespace sleefcu {
namespace gamma64 {
using namespace explog64;

constexpr double LOG2PI_H = 0x1.d67f1c864beb5p-1, LOG2PI_L = -0x1.65b5a1b7ff5dfp-55;   // log(2 pi)/2
constexpr double LOGPI_H = 0x1.250d048e7a1bdp+0, LOGPI_L = 0x1.7abf2ad8d5088p-57;      // log(pi)
constexpr double PI_H = 0x1.921fb54442d18p+1, PI_L = 0x1.1a62633145c07p-53;
// 200 ln 2 as a DD: 200 times the 42-bit head of ln 2 (exact) and RN(200 times its tail)
constexpr double LN2X200_H = 0x1.1542457337bc0p+7, LN2X200_L = 0x1.82e1c6b73c89ep-37;
constexpr uint64_t SIGN = 0x8000000000000000ull;

static __constant__ double kLgR2H[4] = {0x1.b0ee6072093cep-2, 0x1.6c58518ef209cp-58, 0x1.4a34cc4a60fa6p-2, 0x1.1b98b7d24eb82p-56};
static __constant__ double kLgR2P[16] = {
    -0x1.13e001a557606p-4, 0x1.51322ac7d846dp-6, -0x1.e404fc218fc23p-8, 0x1.7add6eadbd405p-9,
    -0x1.38ac5c2b8a199p-10, 0x1.0b36af7f23772p-11, -0x1.d3fd4cdaf22e0p-13, 0x1.a127b9082ca84p-14,
    -0x1.78de521792e56p-15, 0x1.580b6a9b7953fp-16, -0x1.3cb65d569461dp-17, 0x1.25e70a4f871bep-18,
    -0x1.139ba270fa662p-19, 0x1.ffad5d0754437p-21, -0x1.99a8f419f8596p-22, 0x1.7da6d390ec3f8p-24};
static __constant__ double kLgMH[6] = {
    -0x1.eeb95b094c191p-4, -0x1.34022180247c2p-58, 0x1.2aed059bd608ap-5, 0x1.7e1a96f7c7ed0p-63,
    0x1.de9e64df22ef3p-2, -0x1.b1d5ff59dcc8fp-56};
static __constant__ double kLgMP[15] = {
    -0x1.1ae55b180726bp-3, 0x1.e0f840dad650ap-5, -0x1.da59d5374aed9p-6, 0x1.f9ca39da28ed7p-7,
    -0x1.1a8ba4f054ba6p-7, 0x1.456f1b2745dc9p-8, -0x1.7edb81cde7f7cp-9, 0x1.c973218d36f11p-10,
    -0x1.148a003bbd58dp-10, 0x1.51884c3b797c0p-11, -0x1.9f11b5ad1c5d2p-12, 0x1.fea4040bd8d69p-13,
    -0x1.3d5aec9602328p-13, 0x1.bf0b984ee3abdp-14, -0x1.1a86a63641821p-14};
static __constant__ double kLgSt[10] = {
    0x1.5555555555555p-4, -0x1.6c16c16c16c16p-9, 0x1.a01a01a0196bap-11, -0x1.381381362b216p-11,
    0x1.b951df87db260p-11, -0x1.f6a98a1bab42ap-10, 0x1.a3e150e3f70bdp-8, -0x1.dee553034d0abp-6,
    0x1.490abb645435cp-3, -0x1.7031193624fc5p-1};
static __constant__ double kSpH[2] = {-0x1.4abbce625be53p+2, 0x1.05511c684d1cbp-52};
static __constant__ double kSpP[11] = {
    0x1.466bc6775aae2p+1, -0x1.32d2cce62bddep-1, 0x1.50783487f6d9cp-4, -0x1.e3074fec25b1dp-8,
    0x1.e8f4422d6f029p-12, -0x1.6fb6226ceb4fdp-16, 0x1.b1dd7b5e6be80p-21, -0x1.5249d9e04752dp-24,
    0x1.46d5e635ea9dep-23, -0x1.f9b2ef7ed3d1ep-23, 0x1.563183599af6cp-23};

__device__ __forceinline__ d2 neg(d2 a) { return D2(-a.x, -a.y); }

// bounds as bit patterns; the comparisons below are on positive values (or
// on |x|), whose bit order is their value order, so they run on the
// integer pipe
constexpr uint64_t G05 = 0x3FE0000000000000ull, G075 = 0x3FE8000000000000ull, G125 = 0x3FF4000000000000ull;
constexpr uint64_t G175 = 0x3FFC000000000000ull, G25 = 0x4004000000000000ull, G7 = 0x401C000000000000ull;
constexpr uint64_t G8 = 0x4020000000000000ull, G172 = 0x4065800000000000ull, G190 = 0x4067C00000000000ull;
constexpr uint64_t G1015 = 0x7F60000000000000ull, G52 = 0x4330000000000000ull, G60 = 0x43B0000000000000ull;


// lgamma(2 + e), -0.25 <= e < 0.5
__device__ __forceinline__ d2 lg_r2(d2 e) {
  double p = poly_p<16>(e.x, kLgR2P);
  d2 in = add_d2_d(D2(kLgR2H[2], kLgR2H[3]), dmul(e.x, p));
  in = add_d2d2(D2(kLgR2H[0], kLgR2H[1]), mul_d2d2(in, e));
  return mul_d2d2(in, e);
}
// lgamma(1.5 + u), -0.25 <= u < 0.25
__device__ __forceinline__ d2 lg_m(d2 u) {
  double p = poly_p<15>(u.x, kLgMP);
  d2 in = add_d2_d(D2(kLgMH[4], kLgMH[5]), dmul(u.x, p));
  in = add_d2d2(D2(kLgMH[2], kLgMH[3]), mul_d2d2(in, u));
  return add_d2d2(D2(kLgMH[0], kLgMH[1]), mul_d2d2(in, u));
}
// Stirling's form, DD y >= 8
__device__ __forceinline__ d2 lg_stirling(d2 y) {
  d2 ly = logk_dd(y);
  d2 r = mul_d2d2(add_d2_d(y, -0.5), ly);
  r = add_d2d2(r, neg(y));
  // from 2^60 on, log(2 pi)/2 + G(1/y^2)/y < 0.92 is under 2^-12 ulp of the
  // rest (ulp >= 2^13) and is left out (those lanes sort into their own class)
  if (bits(y.x) >= G60) return r;
  r = add_d2d2(r, D2(LOG2PI_H, LOG2PI_L));
  double ry = __ddiv_rn(1.0, y.x);            // one reciprocal: w = 1/y^2 and G(w)/y
  double w = dmul(ry, ry);
  return add_d2_d(r, dmul(poly(w, kLgSt), ry));
}
// lgamma of a DD y > 0; out of line (its four paths are called from the
// positive and the reflected arguments of both functions: one copy of the
// code instead of three, tgamma 2.41 -> 2.48 Gelem/s on GB300, same bits)
static __device__ __noinline__ d2 lgamma_pos(d2 y) {
  const uint64_t b = bits(y.x);                       // y.x > 0 and finite
  if (b >= G8) return lg_stirling(y);
  if (b >= G175 && b < G25) return lg_r2(norm_d2(add_d2_d(y, -2.0)));
  if (b >= G125 && b < G175) return lg_m(norm_d2(add_d2_d(y, -1.5)));
  if (b >= G05 && b < G125) {
    d2 r = b < G075 ? lg_m(norm_d2(add_d2_d(y, -0.5))) : lg_r2(norm_d2(add_d2_d(y, -1.0)));
    return add_d2d2(r, neg(logk_dd(y)));
  }
  int n = int_of(__dsub_rn(8.0, floor(y.x)));         // y + n in [8, 9)
  d2 P = y, z = y;
  for (int i = 1; i < n; i++) {
    z = add_d2_d(z, 1.0);
    P = mul_d2d2(P, z);
  }
  d2 s = lg_stirling(add_d2_d(y, dbl_of(n)));
  return add_d2d2(s, neg(logk_dd(P)));
}
// sin(pi x) as a DD, |x| < 2^52
__device__ __forceinline__ d2 sinpi_dd(double x) {
  double r = __dsub_rn(x, dmul(2.0, drint(dmul(0.5, x))));
  double s = okey(r) > okey(0.5) ? __dsub_rn(1.0, r) : (okey(r) < okey(-0.5) ? __dsub_rn(-1.0, r) : r);
  d2 T = mul_dd(s, s);
  double p = poly_p<11>(T.x, kSpP);
  d2 in = add_d2_d(D2(kSpH[0], kSpH[1]), dmul(T.x, p));
  in = add_d2d2(D2(PI_H, PI_L), mul_d2d2(T, in));
  return mul_d2_d(in, s);
}
// log-gamma as a DD, sign of gamma (finite x, not a non-positive integer)
__device__ __forceinline__ d2 lgamma_dd(double x, int &sign) {
  sign = 1;
  if (gt_0(x)) return lgamma_pos(D2(x, 0.0));
  // |x| < 2^-900: sin(pi x) is pi x to far below an ulp, and pi x itself
  // would lose its precision in the subnormal range; it is formed from
  // x 2^200 (exact) and 200 ln 2 is taken off its logarithm
  bool up = (bits(x) & ABS64) < 0x07B0000000000000ull;          // |x| < 2^-900
  d2 sp = up ? mul_d2_d(D2(PI_H, PI_L), dmul(x, 0x1p200)) : sinpi_dd(x);
  bool negs = lt_0(sp.x);
  sign = negs ? -1 : 1;
  d2 l = logk_dd(D2(fabs(sp.x), negs ? -sp.y : sp.y));
  if (up) l = add_d2d2(l, D2(-LN2X200_H, -LN2X200_L));
  d2 r = add_d2d2(D2(LOGPI_H, LOGPI_L), neg(l));
  d2 g = lgamma_pos(add_dd(1.0, -x));
  return add_d2d2(r, neg(g));
}
// path class for the sorted tiles
__device__ __forceinline__ int gamma_cls(double x) {
  const uint64_t a = bits(x) & ABS64;
  if (a > G1015 || a == 0) return 7;                  // also inf and NaN
  if (bits(x) >> 63) return a >= G7 ? 5 : 6;
  if (a >= G8) return 0;
  if (a >= G175 && a < G25) return 1;
  if (a >= G125 && a < G175) return 2;
  if (a >= G05 && a < G125) return 3;
  return 4;
}
__device__ __forceinline__ bool neg_int(double x) {   // x < 0 and an integer (-inf included)
  const uint64_t a = bits(x) & ABS64;
  return (bits(x) >> 63) && a - 1 < EXP64 && (a >= G52 || integral_b(a));
}

struct LgammaU10 {
  static constexpr int NCLS = 9;
  static constexpr int SORT_EPT = 16;   // 4096-element tiles: nine classes, several of them small
  static constexpr int MIN_BLOCKS = 4;  // 64 registers: four 256-thread blocks per SM
  // class 8: x >= 2^60, Stirling's form without its two smallest terms
  __device__ static int cls(double x) {
    const int c = gamma_cls(x);
    return (c == 0 && bits(x) >= G60) ? 8 : c;
  }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    if (is_nan_b(bx)) return from_bits(QNAN64);
    if ((bx & ABS64) == INF || (bx & ABS64) == 0 || neg_int(x) || (!(bx >> 63) && bx > G1015))
      return from_bits(INF);
    int sign;
    d2 L = lgamma_dd(x, sign);
    double y = __dadd_rn(L.x, L.y);
    if ((bits(y) & ABS64) >= INF) y = from_bits(INF);
    return canon(y);
  }
};
// y 2^k for a positive normal y: the exponent field when the result is
// normal, +inf above, two multiplications by normal powers of two (one
// rounding) below
__device__ __forceinline__ double scale2_any(double y, int k) {
  const int e = (int)(bits(y) >> 52) - 1023 + k;
  if (e > 1023) return from_bits(INF);
  if (e >= -1022) return from_bits(bits(y) + ((uint64_t)(int64_t)k << 52));
  const int k1 = k / 2, k2 = k - k1;
  return dmul(dmul(y, pow2i(k1)), pow2i(k2));
}
constexpr uint64_t G2M900 = 0x07B0000000000000ull;   // 2^-900

struct TgammaU10 {
  static constexpr int NCLS = 8;
  static constexpr int SORT_EPT = 16;   // 4096-element tiles: eight classes, several of them small
  static constexpr int MIN_BLOCKS = 4;  // 64 registers: four 256-thread blocks per SM
  __device__ static int cls(double x) { return gamma_cls(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    if (is_nan_b(bx) || bx == (INF | SIGN) || neg_int(x)) return from_bits(QNAN64);
    if ((bx & ABS64) == 0) return from_bits(INF | (bx & SIGN));
    if (!(bx >> 63) && bx > G172) return from_bits(INF);
    if ((bx >> 63) && (bx & ABS64) > G190) return lt_0(sinpi_dd(x).x) ? -0.0 : 0.0;
    if (gt_0(x)) return canon(expk(lgamma_pos(D2(x, 0.0))));
    // x < 0: the reflection in linear form, gamma(x) = pi / (sin(pi x) e^g)
    // with g = lgamma(1 - x), e^-g = 2^k (1 + s) from the DD exp core; for
    // |x| < 2^-900 sin(pi x) = pi x is formed from x 2^200 (full precision
    // where pi x would be subnormal) and 2^-200 rejoins 2^k
    const int up = (bx & ABS64) < G2M900 ? 200 : 0;
    d2 sp = up ? mul_d2_d(D2(PI_H, PI_L), dmul(x, 0x1p200)) : sinpi_dd(x);
    const bool negs = lt_0(sp.x);
    d2 d = D2(fabs(sp.x), negs ? -sp.y : sp.y);
    d2 g = lgamma_pos(add_dd(1.0, -x));
    double k;
    d2 e = add_d_d2_fast(1.0, expk_s(D2(-g.x, -g.y), k));
    d2 q = div_d2d2(mul_d2d2(D2(PI_H, PI_L), e), d);
    double y = scale2_any(__dadd_rn(q.x, q.y), int_of(k) + up);
    return canon(negs ? -y : y);
  }
};

}  // namespace gamma64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define SORTED64(NAME, F)                                                                   \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_sorted64<gamma64::F>("sleefcu_" #NAME, x, out, n, s);                     \
  }
#define SORTED64_MASKED(NAME, F)                                                    \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<gamma64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
SORTED64(tgamma_u10_f64, TgammaU10)
SORTED64_MASKED(tgamma_u10_f64, TgammaU10)
SORTED64(tgamma_u35_f64, TgammaU10)
SORTED64_MASKED(tgamma_u35_f64, TgammaU10)
SORTED64(lgamma_u10_f64, LgammaU10)
SORTED64_MASKED(lgamma_u10_f64, LgammaU10)
SORTED64(lgamma_u35_f64, LgammaU10)
SORTED64_MASKED(lgamma_u35_f64, LgammaU10)
#undef SORTED64
#undef SORTED64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
