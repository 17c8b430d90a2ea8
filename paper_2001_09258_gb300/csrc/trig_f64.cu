// FP64 sin, cos, tan, sincos (u10 and u35) for sm_103a.
//
// Method (Sections 5.1, 5.2, 5.8 and Appendix A of the paper):
//   |x| < 15    level-1 Cody-Waite: x - q pi/2 with the two-constant split of
//               pi/2 printed in the tan listing (fma with the head, DD add of
//               the tail);
//   |x| < 1e14  level-2 Cody-Waite: head by fma (exact for these q), second
//               constant by an exact DD product, third constant into the tail;
//   otherwise   the vectorizable Payne-Hanek reduction (Eq. 1 in DD over the
//               four table words of the Payne-Hanek table-generation figure).
// Each lane takes the reduction its own |x| calls for (the paper's
// bit-consistent variant, Section 4: small-argument method first, the next
// method only for elements it does not cover); a warp runs a reduction only
// if one of its lanes needs it.  Classification, quadrant bookkeeping, signs
// and special values run on the integer pipe, leaving the FP64 pipe (the
// bound of this family on GB300) to the arithmetic of the method.
#include "sleefcu_common.cuh"
#include "sleefcu_phtab.inc"

namespace sleefcu {
namespace trig64 {

constexpr double PIO2_A = 0x1.921fb54442d18p0;    // Appendix A listing
constexpr double PIO2_B = 0x1.1a62633145c07p-54;  // Appendix A listing
constexpr double PIO2_C = -0x1.f1976b7ed8fbcp-110;
constexpr double TWOPI_H = 0x1.921fb54442d18p2;   // Appendix A listing
constexpr double TWOPI_L = 0x1.1a62633145c07p-52;
constexpr double R_1_PI = 0x1.45f306dc9c883p-2;
constexpr double R_2_PI = 0x1.45f306dc9c883p-1;
constexpr uint64_t B15 = 0x402e000000000000ull;   // bits of 15.0
constexpr uint64_t B1 = 0x3ff0000000000000ull;    // bits of 1.0
constexpr uint64_t B1E14 = 0x42d6bcc41e900000ull; // bits of 1e14

static __constant__ double kSinU10[7] = {
  0x1.111111111109fp-7, -0x1.a01a01a0129ddp-13, 0x1.71de3a51b383dp-19,
  -0x1.ae64546a1a9ebp-26, 0x1.6123b2c07aaa7p-33, -0x1.ae3cc8078333ap-41,
  0x1.877f977ffe028p-49};
constexpr double SIN_C1H = -0x1.5555555555555p-3, SIN_C1L = 0x1.07fb00106bcfdp-57;
static __constant__ double kSinU35[8] = {
  -0x1.5555555555555p-3, 0x1.11111111110bdp-7, -0x1.a01a01a013e17p-13,
  0x1.71de3a5220856p-19, -0x1.ae645492b5795p-26, 0x1.6123bb419f3c8p-33,
  -0x1.ae3ea885fb135p-41, 0x1.87ab1397c30b7p-49};
// Appendix A tan listing, constant term first
static __constant__ double kTanC[8] = {
  0x1.111111110e933p-3, 0x1.ba1ba1bdcec06p-5, 0x1.664f4729f98e5p-6,
  0x1.226e7bfa35090p-7, 0x1.d6c27c371c959p-9, 0x1.7eef631e20b93p-10,
  0x1.269be400de3afp-11, 0x1.5445f555134edp-12};
constexpr double TAN_C3 = 0x1.5555555555568p-2;
constexpr double SC_S1H = -0x1.5555555555543p-3, SC_S1L = 0x1.cc5eebaea7e3cp-57;
static __constant__ double kScSU10[5] = {
  0x1.111111110eea5p-7, -0x1.a01a019ad6669p-13, 0x1.71de3466b0f92p-19,
  -0x1.ae5d912c0cb21p-26, 0x1.5d558cd2a4be1p-33};
static __constant__ double kScC[6] = {
  0x1.5555555555546p-5, -0x1.6c16c16c14555p-10, 0x1.a01a019b8491fp-16,
  -0x1.27e4f73296656p-22, 0x1.1ee95b26826a1p-29, -0x1.8f6489336e5adp-37};
static __constant__ double kScSU35[6] = {
  -0x1.5555555555543p-3, 0x1.111111110ef1dp-7, -0x1.a01a019ae1837p-13,
  0x1.71de346e3d979p-19, -0x1.ae5d95f8b7e3ep-26, 0x1.5d56b550f4cf7p-33};

// ---------------- reductions ----------------
__device__ __forceinline__ d2 cw1(double x, double qd) {
  double u = __fma_rn(qd, -PIO2_A, x);
  return add_dd_fast(u, dmul(qd, -PIO2_B));
}
// cos at |x| < 1 (q = +-1): the fma head is not exact there, so q A is an
// exact DD product added with TwoSum
__device__ __forceinline__ d2 cw1_exact(double x, double qd) {
  d2 s = add_d_d2(x, mul_dd(qd, -PIO2_A));
  return add_d2_d_fast(s, dmul(qd, -PIO2_B));
}
__device__ __forceinline__ d2 cw2(double x, double qd) {
  double u = __fma_rn(qd, -PIO2_A, x);
  d2 h = mul_dd(qd, -PIO2_B);
  d2 s = add_d_d2(u, h);
  s.y = __fma_rn(qd, -PIO2_C, s.y);
  return s;
}
__device__ __forceinline__ double cw1_d(double x, double qd) {
  return __fma_rn(qd, -PIO2_B, __fma_rn(qd, -PIO2_A, x));
}
__device__ __forceinline__ double cw2_d(double x, double qd) {
  return __fma_rn(qd, -PIO2_C, __fma_rn(qd, -PIO2_B, __fma_rn(qd, -PIO2_A, x)));
}

// one rfrac step of Eq. (1): r = rint(4 x.x) quarter turns, kept mod 4 in q
__device__ __forceinline__ void ph_step(d2 &x, int &q) {
  double r = drint(dmul(4.0, x.x));
  q += low2_of_int(r);
  x.x = __fma_rn(r, -0.25, x.x);
  x = norm_d2(x);
}

// Payne-Hanek (Section 5.8): returns s in [-pi/4, pi/4] as DD and the
// quarter-turn count mod 4.  Only lanes with |d| >= 1e14 or non-finite d
// call it.  The table drops M*I(E)/2 turns: a half turn is restored through
// q when the mantissa and I(E) are odd.
static __device__ __noinline__ d2 ph(double d, int &q) {
  uint64_t b = bits(d);
  bool fin = is_finite_b(b);
  uint64_t bf = fin ? b : 0;
  int e = (int)((bf >> 52) & 0x7FF) - 1023;
  int sh = e > 700 ? 130 : 2;
  int ex = min(max(e, 0), 1023);
  checked_note(fin && ex != e);       // a finite argument below 1e14 never comes here
  double u = bf ? from_bits(bf - ((uint64_t)sh << 52)) : 0.0;   // d * 2^-sh, exact
  const double2 *T = reinterpret_cast<const double2 *>(k_phtab64 + 4 * ex);
  double2 ta = __ldg(T), tb = __ldg(T + 1);
  int qq = 0;
  d2 x = mul_dd(u, ta.x);          // (0,0) + y is y exactly: the first add is skipped
  ph_step(x, qq);
  x = add_d2d2(x, mul_dd(u, ta.y));
  ph_step(x, qq);
  x = add_d2d2(x, mul_dd(u, tb.x));
  ph_step(x, qq);
  x = add_d2d2(x, mul_dd(u, tb.y));
  ph_step(x, qq);
  x = mul_d2d2(x, D2(TWOPI_H, TWOPI_L));
  uint32_t ib = (__ldg(k_phbit64 + (ex >> 5)) >> (ex & 31)) & 1u;
  q = (qq + 2 * (int)((uint32_t)bf & ib)) & 3;
  if (!fin) x.x = from_bits(QNAN64);
  return x;
}

// move a quarter-turn result of the wrong parity by +-pi/2 onto the
// half-turn grid of the sine polynomial (parity 0: sin, 1: cos)
__device__ __forceinline__ d2 ph_fold(d2 r, int &q, int parity) {
  if ((q & 1) != parity) {
    bool ge = r.x >= 0.0;
    double sa = ge ? -PIO2_A : PIO2_A, sb = ge ? -PIO2_B : PIO2_B;
    r = add_d2d2_fast(D2(sa, sb), r);
    q = (q + (ge ? 1 : -1)) & 3;
  }
  return r;
}

// half-turn reduction: parity 0 gives q even (sin), 1 gives q odd (cos)
template <int PARITY>
__device__ __forceinline__ d2 reduce_half(double x, uint64_t ab, int &q) {
  if (ab < B1E14) {
    double k, qd;
    if (PARITY == 0) {
      k = drint(dmul(x, R_1_PI));
      qd = __dadd_rn(k, k);
      q = (low2_of_int(k) << 1) & 3;
    } else {
      k = drint(__fma_rn(x, R_1_PI, -0.5));
      qd = __fma_rn(2.0, k, 1.0);
      q = ((low2_of_int(k) << 1) + 1) & 3;
      if (ab < B1) return cw1_exact(x, qd);
    }
    if (ab < B15) return cw1(x, qd);
    return cw2(x, qd);
  }
  d2 r = ph(x, q);
  return ph_fold(r, q, PARITY);
}
template <int PARITY>
__device__ __forceinline__ double reduce_half_d(double x, uint64_t ab, int &q) {
  if (ab < B1E14) {
    double k, qd;
    if (PARITY == 0) {
      k = drint(dmul(x, R_1_PI));
      qd = __dadd_rn(k, k);
      q = (low2_of_int(k) << 1) & 3;
    } else {
      k = drint(__fma_rn(x, R_1_PI, -0.5));
      qd = __fma_rn(2.0, k, 1.0);
      q = ((low2_of_int(k) << 1) + 1) & 3;
    }
    if (ab < B15) return cw1_d(x, qd);
    return cw2_d(x, qd);
  }
  d2 r = ph(x, q);
  r = ph_fold(r, q, PARITY);
  return __dadd_rn(r.x, r.y);
}
__device__ __forceinline__ d2 reduce_quarter(double x, uint64_t ab, int &q) {
  if (ab < B1E14) {
    double qd = drint(dmul(x, R_2_PI));
    q = low2_of_int(qd);
    if (ab < B15) return cw1(x, qd);
    return cw2(x, qd);
  }
  return ph(x, q);
}
__device__ __forceinline__ double reduce_quarter_d(double x, uint64_t ab, int &q) {
  if (ab < B1E14) {
    double qd = drint(dmul(x, R_2_PI));
    q = low2_of_int(qd);
    if (ab < B15) return cw1_d(x, qd);
    return cw2_d(x, qd);
  }
  d2 r = ph(x, q);
  return __dadd_rn(r.x, r.y);
}

// reduction path of an argument: 0 level-1 Cody-Waite, 1 level-2, 2 Payne-Hanek
// (|x| >= 1e14, infinities and NaN)
__device__ __forceinline__ int path_of(double x) {
  uint64_t ab = bits(x) & ABS64;
  return ab < B15 ? 0 : (ab < B1E14 ? 1 : 2);
}
#define TRIG_PATHS                       \
  static constexpr int NCLS = 3;         \
  __device__ static int cls(double x) { return path_of(x); }
// cos u10 has a fourth path: the exact head for |x| < 1
#define COS_PATHS                        \
  static constexpr int NCLS = 4;         \
  __device__ static int cls(double x) {  \
    return (bits(x) & ABS64) < B1 ? 3 : path_of(x); }

// ---------------- polynomials ----------------
// sin s = s + s t (c1 + t P(t)), t = s^2, the leading products in DD
__device__ __forceinline__ double sin_poly_u10(d2 s) {
  d2 t = sqr_d2(s);
  double p = poly(t.x, kSinU10);
  d2 w = add_d2_d_fast(D2(SIN_C1H, SIN_C1L), dmul(t.x, p));
  w = mul_d2d2(t, w);
  w = mul_d2d2(s, w);
  d2 r = add_d2d2_fast(s, w);
  return __dadd_rn(r.x, r.y);
}
__device__ __forceinline__ double sin_poly_u35(double s) {
  double t = dmul(s, s);
  return __fma_rn(dmul(s, t), poly(t, kSinU35), s);
}

struct SinU10 {
  TRIG_PATHS
  __device__ double operator()(double x) const {
    uint64_t ab = bits(x) & ABS64;
    int q;
    d2 s = reduce_half<0>(x, ab, q);
    double y = neg_if(sin_poly_u10(s), q & 2);
    if (ab == 0) y = x;
    return canon(y);
  }
};
struct CosU10 {
  COS_PATHS
  __device__ double operator()(double x) const {
    uint64_t ab = bits(x) & ABS64;
    int q;
    d2 s = reduce_half<1>(x, ab, q);
    return canon(neg_if(sin_poly_u10(s), !(q & 2)));
  }
};
struct SinU35 {
  TRIG_PATHS
  __device__ double operator()(double x) const {
    uint64_t ab = bits(x) & ABS64;
    int q;
    double s = reduce_half_d<0>(x, ab, q);
    double y = neg_if(sin_poly_u35(s), q & 2);
    if (ab == 0) y = x;
    return canon(y);
  }
};
struct CosU35 {
  TRIG_PATHS
  __device__ double operator()(double x) const {
    uint64_t ab = bits(x) & ABS64;
    int q;
    double s = reduce_half_d<1>(x, ab, q);
    return canon(neg_if(sin_poly_u35(s), !(q & 2)));
  }
};

// tan: Appendix A listing with the level-2 Cody-Waite added
struct TanU10 {
  TRIG_PATHS
  __device__ double operator()(double d) const {
    uint64_t ab = bits(d) & ABS64;
    int q;
    d2 x = reduce_quarter(d, ab, q), y;
    y = scale_d2(x, 0.5);
    x = sqr_d2(y);
    double u = poly(x.x, kTanC);
    u = __fma_rn(u, x.x, TAN_C3);
    x = add_d2d2_fast(y, mul_d2_d(mul_d2d2(x, y), u));
    y = add_d_d2_fast(-1.0, sqr_d2(x));
    x = scale_d2(x, -2.0);
    if (q & 1) {
      d2 t = x;
      x = y;
      y = D2(-t.x, -t.y);
    }
    x = div_d2d2(x, y);
    double r = __dadd_rn(x.x, x.y);
    if (ab == 0) r = d;
    return canon(r);
  }
};
// a / b within about a unit of the correctly rounded quotient: the
// reciprocal of b's significand from the binary32 reciprocal (significand
// truncated to 24 bits, widened exactly) and two Newton steps with fma,
// scaled by 2^-ilogb|b|, then q = a r and one fma correction q + (a - q b) r:
// six FP64-pipe operations and a software multiply instead of a correctly
// rounded division; b outside [2^-1000, 2^1000] takes the IEEE division
__device__ __forceinline__ double div_u35(double a, double b) {
  const uint64_t bb = bits(b) & ABS64;
  if (!(bb >= 0x0170000000000000ull && bb <= 0x7E70000000000000ull)) return __ddiv_rn(a, b);
  const uint64_t man = bb & 0x000FFFFFFFFFFFFFull;
  const int e = (int)(bb >> 52) - 1023;
  const double m = from_bits(0x3FF0000000000000ull | man);
  const uint32_t rb = fbits(__frcp_rn(from_fbits(0x3F800000u | (uint32_t)(man >> 29))));
  double y = from_bits(((uint64_t)((rb >> 23) + 896) << 52) | ((uint64_t)(rb & 0x7FFFFFu) << 29));
  double t = __fma_rn(-m, y, 1.0);
  y = __fma_rn(y, t, y);
  t = __fma_rn(-m, y, 1.0);
  y = __fma_rn(y, t, y);                                       // 1/m to about an ulp
  const double r = neg_if(from_bits(bits(y) - ((uint64_t)(int64_t)e << 52)), (bits(b) >> 63) != 0);
  const double q = dmul(a, r);
  return __fma_rn(__fma_rn(-q, b, a), r, q);
}

struct TanU35 {
  TRIG_PATHS
  __device__ double operator()(double d) const {
    uint64_t ab = bits(d) & ABS64;
    int q;
    double s = reduce_quarter_d(d, ab, q);
    double y = dmul(s, 0.5), t = dmul(y, y);
    double u = __fma_rn(poly(t, kTanC), t, TAN_C3);
    double tt = __fma_rn(dmul(y, t), u, y);
    double num = __dadd_rn(tt, tt), den = __fma_rn(-tt, tt, 1.0);
    double r = (q & 1) ? div_u35(-den, num) : div_u35(num, den);
    if (ab == 0) r = d;
    return canon(r);
  }
};

__device__ __forceinline__ void sc_quadrant(int q, double &sn, double &cs) {
  if (q & 1) {
    double t = sn;
    sn = cs;
    cs = -t;
  }
  if (q & 2) {
    sn = -sn;
    cs = -cs;
  }
}

struct SinCosU10 {
  TRIG_PATHS
  __device__ void operator()(double d, double &os, double &oc) const { dual(d, os, oc); }
  __device__ void dual(double d, double &os, double &oc) const {
    uint64_t ab = bits(d) & ABS64;
    int q;
    d2 s = reduce_quarter(d, ab, q);
    d2 t = sqr_d2(s);
    double p = poly(t.x, kScSU10);
    d2 w = add_d2_d_fast(D2(SC_S1H, SC_S1L), dmul(t.x, p));
    w = mul_d2d2(t, w);
    w = mul_d2d2(s, w);
    d2 rs = add_d2d2_fast(s, w);
    double sn = __dadd_rn(rs.x, rs.y);
    double pc = poly(t.x, kScC);
    d2 h = add_d_d2_fast(1.0, scale_d2(t, -0.5));
    h = add_d2_d_fast(h, dmul(dmul(t.x, t.x), pc));
    double cs = __dadd_rn(h.x, h.y);
    sc_quadrant(q, sn, cs);
    if (ab == 0) sn = d;
    os = canon(sn);
    oc = canon(cs);
  }
};
struct SinCosU35 {
  TRIG_PATHS
  __device__ void operator()(double d, double &os, double &oc) const { dual(d, os, oc); }
  __device__ void dual(double d, double &os, double &oc) const {
    uint64_t ab = bits(d) & ABS64;
    int q;
    double s = reduce_quarter_d(d, ab, q);
    double t = dmul(s, s);
    double sn = __fma_rn(dmul(s, t), poly(t, kScSU35), s);
    double cs = __fma_rn(t, __fma_rn(t, poly(t, kScC), -0.5), 1.0);
    sc_quadrant(q, sn, cs);
    if (ab == 0) sn = d;
    os = canon(sn);
    oc = canon(cs);
  }
};

}  // namespace trig64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define UNARY64(NAME, F)                                                                    \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_sorted64<trig64::F>("sleefcu_" #NAME, x, out, n, s);                       \
  }
#define UNARY64_MASKED(NAME, F)                                                     \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<trig64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
UNARY64(sin_u10_f64, SinU10)
UNARY64_MASKED(sin_u10_f64, SinU10)
UNARY64(sin_u35_f64, SinU35)
UNARY64_MASKED(sin_u35_f64, SinU35)
UNARY64(cos_u10_f64, CosU10)
UNARY64_MASKED(cos_u10_f64, CosU10)
UNARY64(cos_u35_f64, CosU35)
UNARY64_MASKED(cos_u35_f64, CosU35)
UNARY64(tan_u10_f64, TanU10)
UNARY64_MASKED(tan_u10_f64, TanU10)
UNARY64(tan_u35_f64, TanU35)
UNARY64_MASKED(tan_u35_f64, TanU35)

extern "C" sleefcu_status sleefcu_sincos_u10_f64(const double *x, double *os, double *oc, size_t n,
                                                 sleefcu_stream s) {
  return launch_sorted64_dual<trig64::SinCosU10>("sleefcu_sincos_u10_f64", x, os, oc, n, s);
}
extern "C" sleefcu_status sleefcu_sincos_u35_f64(const double *x, double *os, double *oc, size_t n,
                                                 sleefcu_stream s) {
  return launch_sorted64_dual<trig64::SinCosU35>("sleefcu_sincos_u35_f64", x, os, oc, n, s);
}
extern "C" sleefcu_status sleefcu_sincos_u10_f64_masked(const double *x, const uint8_t *mask, double *os,
                                                        double *oc, size_t n, sleefcu_stream s) {
  return launch_masked64_dual<trig64::SinCosU10>("sleefcu_sincos_u10_f64_masked", x, mask, os, oc, n, s);
}
extern "C" sleefcu_status sleefcu_sincos_u35_f64_masked(const double *x, const uint8_t *mask, double *os,
                                                        double *oc, size_t n, sleefcu_stream s) {
  return launch_masked64_dual<trig64::SinCosU35>("sleefcu_sincos_u35_f64_masked", x, mask, os, oc, n, s);
}
#undef UNARY64
#undef UNARY64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
