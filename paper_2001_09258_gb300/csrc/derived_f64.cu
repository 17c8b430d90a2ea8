// FP64 functions built on the exp/log cores (u10 and u35) for sm_103a:
// exp2, exp10, expm1, log2, log10, log1p, cbrt, sinh, cosh, tanh, asinh,
// acosh, atanh, erf, erfc.  The paper lists them in the library without giving their
// steps; each one here is a short fixed sequence of IEEE operations (DD where
// the 1-ULP bound needs it, Section 3) on top of the Section 5.5-5.7 cores:
//
//   exp2   k = rint(x), r = x - k exact, r ln2 as a DD, the exp tail
//   exp10  k = rint(x log2 10), r = x - k log10(2) (two-part constant, exact
//          head), r ln10 as a DD, the exp tail
//   expm1  2^k s + (2^k - 1) with s = e^r - 1 as a DD and 2^k - 1 an exact DD
//   log2, log10, log1p   log of a DD argument (1 + x exact for log1p), then
//          DD constants (u10) or the core rounded and one fma (u35)
//   cbrt   a in [1, 8) with x = a 2^(3q); a^(-1/3) from a polynomial and one
//          division-free Newton step, y = a z^2, one Newton step on y with
//          y^3 - a in DD (u10) or by one fma (u35)
//   sinh = (e + e/(1+e))/2, cosh = (E + 1/E)/2, tanh = e2/(e2 + 2) with
//          e = e^|x| - 1 and e2 = e^(2|x|) - 1 in DD; e^|x|/2 for |x| > 22
//   asinh, acosh, atanh   log of |x| + sqrt(x^2+1), x + sqrt((x-1)(x+1)),
//          (1+|x|)/(1-|x|), each argument a DD
//
// Special values follow C99 Annex F (Section 5.10); NaN results are the
// canonical quiet NaN.  The branches taken by rare lanes (huge arguments,
// the large-|x| hyperbolic path) change no bit of the other lanes' results.
#include "explog64_core.cuh"

namespace sleefcu {
namespace derived64 {
using namespace explog64;

constexpr double RL2H = 0x1.71547652b82fep+0, RL2L = 0x1.777d0ffda0d24p-56;     // 1/ln2
constexpr double RL10H = 0x1.bcb7b1526e50ep-2, RL10L = 0x1.95355baaafad3p-57;   // 1/ln10
constexpr double LN10H = 0x1.26bb1bbb55516p+1, LN10L = -0x1.f48ad494ea3e9p-53;  // ln10
constexpr double LOG2_10 = 0x1.a934f0979a371p+1;
constexpr double L10A = 0x1.34413509f79ffp-2, L10B = -0x1.9dc1da994fd21p-59;    // log10(2)
constexpr double LG2H = 0x1.34413509f7800p-2, LG2L = 0x1.fef311f12b358p-46;     // 42-bit head
constexpr double THIRD = 0x1.5555555555555p-2;
constexpr double CBRT_C1 = 0x1.965fea53d6e3dp-1, CBRT_C2 = 0x1.428a2f98d728bp-1; // 2^(-1/3), 2^(-2/3)
constexpr uint64_t SIGN = 0x8000000000000000ull;
constexpr uint64_t B1100 = 0x4091300000000000ull;   // 1100.0
constexpr uint64_t B350 = 0x4075E00000000000ull;    // 350.0
constexpr uint64_t B711 = 0x4086380000000000ull;    // 711.0
constexpr uint64_t B20 = 0x4034000000000000ull;     // 20.0
constexpr uint64_t BM28 = 0x3E30000000000000ull;    // 2^-28
constexpr uint64_t ONE = 0x3FF0000000000000ull;

static __constant__ double kExpm1U35[10] = {
  0x1.0000000000005p-1, 0x1.5555555555539p-3, 0x1.555555555228ep-5, 0x1.1111111119010p-7,
  0x1.6c16c17ee7257p-10, 0x1.a01a0174fb45ep-13, 0x1.a019a74a758d7p-16, 0x1.71de882490dc7p-19,
  0x1.28a2068fa4cf1p-22, 0x1.ae6bacbadab12p-26};
static __constant__ double kCbrt[8] = {
  0x1.bf45ec441bd23p-1, -0x1.8d93481324a0ap-3, 0x1.6176914abb262p-4, -0x1.6ea83723fc3a3p-5,
  0x1.925bc75c45e3cp-6, -0x1.cda96200ffa66p-7, 0x1.5223d83416936p-7, -0x1.a6ef2b72239f2p-8};

__device__ __forceinline__ double copysign_b(double y, uint64_t bx) {
  return from_bits((bits(y) & ABS64) | (bx & SIGN));
}
// e^t - 1 for |t| <= ln2/2, polynomial fitted relative to e^t - 1, one rounding
__device__ __forceinline__ double em1_r_u35(double t) {
  return __fma_rn(dmul(t, t), poly(t, kExpm1U35), t);
}
// 2^k s + (2^k - 1) as a DD (k <= 1000), 2^k - 1 formed exactly by TwoSum
__device__ __forceinline__ d2 em1_join(d2 s, double k) {
  double p = pow2i(int_of(k));
  return add_d2d2(add_dd(p, -1.0), scale_d2(s, p));
}
// k and e^r - 1 in double for the u35 forms
__device__ __forceinline__ double em1_u35(double xc, double &k) {
  k = drint(dmul(xc, R_LN2));
  double r = __fma_rn(k, -L2B, __fma_rn(k, -L2A, xc));
  return em1_r_u35(r);
}
// log of a DD a > 0 as a DD
__device__ __forceinline__ d2 log_dd(d2 a) {
  int e;
  d2 lm = logm_u10(a, e);
  double ed = dbl_of(e);
  return add_d2d2(D2(dmul(ed, L2H), dmul(ed, L2L)), lm);
}

// ---------------- exp2, exp10 ----------------
__device__ __forceinline__ double exp_out(uint64_t b, bool inr, double y) {
  if (!inr) y = is_nan_b(b) ? from_bits(QNAN64) : ((b >> 63) ? 0.0 : from_bits(INF));
  return canon(y);
}
struct Exp2U10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B1100;
    double xc = inr ? x : 0.0;
    double k = drint(xc);
    d2 t = mul_d2_d(D2(L2A, L2B), __dsub_rn(xc, k));
    return exp_out(b, inr, exp_tail_u10(t.x, t.y, int_of(k)));
  }
};
struct Exp2U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B1100;
    double xc = inr ? x : 0.0;
    double k = drint(xc);
    double t = dmul(__dsub_rn(xc, k), L2A);
    return exp_out(b, inr, scale2(__dadd_rn(1.0, em1_r_u35(t)), int_of(k)));
  }
};
struct Exp10U10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B350;
    double xc = inr ? x : 0.0;
    double k = drint(dmul(xc, LOG2_10));
    double h = __fma_rn(k, -L10A, xc);
    double r = __fma_rn(k, -L10B, h);
    double rl = __fma_rn(k, -L10B, __dsub_rn(h, r));
    d2 t = mul_d2d2(D2(r, rl), D2(LN10H, LN10L));
    return exp_out(b, inr, exp_tail_u10(t.x, t.y, int_of(k)));
  }
};
struct Exp10U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B350;
    double xc = inr ? x : 0.0;
    double k = drint(dmul(xc, LOG2_10));
    double r = __fma_rn(k, -L10B, __fma_rn(k, -L10A, xc));
    return exp_out(b, inr, scale2(__dadd_rn(1.0, em1_r_u35(dmul(r, LN10H))), int_of(k)));
  }
};

// ---------------- expm1 ----------------
__device__ __forceinline__ double expm1_out(double x, double y) {
  bool inr = gt_c(x, -40.0) && lt_c(x, 710.0);
  if (eq_0(x)) y = x;
  if (!inr) y = ge_c(x, 710.0) ? from_bits(INF) : (le_c(x, -40.0) ? -1.0 : from_bits(QNAN64));
  return canon(y);
}
struct Expm1U10 {
  __device__ double operator()(double x) const {
    double xc = (gt_c(x, -40.0) && lt_c(x, 710.0)) ? x : 0.0;
    double k;
    d2 s = expk_s(D2(xc, 0.0), k);
    double y;
    if (int_of(k) > 1000) {
      d2 e = add_d_d2_fast(1.0, s);
      y = scale2(__dadd_rn(e.x, e.y), int_of(k));
    } else {
      d2 r = em1_join(s, k);
      y = __dadd_rn(r.x, r.y);
    }
    return expm1_out(x, y);
  }
};
struct Expm1U35 {
  __device__ double operator()(double x) const {
    double xc = (gt_c(x, -40.0) && lt_c(x, 710.0)) ? x : 0.0;
    double k;
    double v = em1_u35(xc, k);
    double y;
    if (int_of(k) > 1000) {
      y = scale2(__dadd_rn(1.0, v), int_of(k));
    } else {
      double p = pow2i(int_of(k));
      y = __fma_rn(p, v, __dsub_rn(p, 1.0));
    }
    return expm1_out(x, y);
  }
};

// ---------------- log2, log10, log1p ----------------
__device__ __forceinline__ double log_out(uint64_t b, double y) {
  if ((b & ABS64) == 0) return from_bits(0xFFF0000000000000ull);
  if ((b >> 63) || is_nan_b(b)) return from_bits(QNAN64);
  if (b == INF) return from_bits(INF);
  return canon(y);
}
__device__ __forceinline__ double log_arg(uint64_t b) {
  return (b - 1) < DMAX ? from_bits(b) : 1.0;      // finite and > 0, else 1
}
struct Log2U10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    int e;
    d2 lm = logm_u10(D2(log_arg(b), 0.0), e);
    d2 p = mul_d2d2(lm, D2(RL2H, RL2L));
    d2 r = add_d_d2(dbl_of(e), p);
    return log_out(b, __dadd_rn(r.x, r.y));
  }
};
struct Log2U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    int e;
    d2 lm = logm_u10(D2(log_arg(b), 0.0), e);
    return log_out(b, __fma_rn(__dadd_rn(lm.x, lm.y), RL2H, dbl_of(e)));
  }
};
struct Log10U10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    int e;
    d2 lm = logm_u10(D2(log_arg(b), 0.0), e);
    d2 p = mul_d2d2(lm, D2(RL10H, RL10L));
    double ed = dbl_of(e);
    d2 r = add_d2d2(D2(dmul(ed, LG2H), dmul(ed, LG2L)), p);
    return log_out(b, __dadd_rn(r.x, r.y));
  }
};
struct Log10U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    int e;
    d2 lm = logm_u10(D2(log_arg(b), 0.0), e);
    return log_out(b, __fma_rn(dbl_of(e), L10A, dmul(__dadd_rn(lm.x, lm.y), RL10H)));
  }
};
__device__ __forceinline__ double log1p_out(double x, double y) {
  uint64_t b = bits(x), ab = b & ABS64;
  if (b == (SIGN | ONE)) return from_bits(0xFFF0000000000000ull);       // x = -1
  if (((b >> 63) && ab > ONE) || ab > EXP64) return from_bits(QNAN64);  // x < -1 or NaN
  if (b == INF) return from_bits(INF);
  if (ab == 0) return x;
  return canon(y);
}
__device__ __forceinline__ double log1p_arg(double x) {
  uint64_t b = bits(x), ab = b & ABS64;
  return (!((b >> 63) && ab >= ONE) && ab <= DMAX) ? x : 0.0;           // -1 < x < inf
}
struct Log1pU10 {
  __device__ double operator()(double x) const {
    d2 r = log_dd(add_dd(1.0, log1p_arg(x)));
    return log1p_out(x, __dadd_rn(r.x, r.y));
  }
};
struct Log1pU35 {
  __device__ double operator()(double x) const {
    int e;
    double lm = logm_u35(add_dd(1.0, log1p_arg(x)), e);
    return log1p_out(x, __fma_rn(dbl_of(e), L2A, lm));
  }
};

// ---------------- cbrt ----------------
template <bool U10>
__device__ __forceinline__ double cbrt_core(double x) {
  uint64_t bx = bits(x), ab = bx & ABS64;
  bool fin = ab - 1 < INF - 1;                     // finite and non-zero
  double a0 = fin ? from_bits(ab) : 1.0;
  int off = 0;
  if (bits(a0) < 0x0010000000000000ull) { a0 = dmul(a0, 0x1p54); off = 18; }   // a0 > 0
  uint64_t b0 = bits(a0);
  int e = (int)(b0 >> 52) - 1023;
  int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  int i = e - 3 * q;
  double m = from_bits((b0 & 0x000FFFFFFFFFFFFFull) | ONE);     // [1, 2)
  double a = dmul(m, pow2i(i));                             // [1, 8)
  double c = i == 0 ? 1.0 : (i == 1 ? CBRT_C1 : CBRT_C2);
  double z = dmul(poly(__dsub_rn(m, 1.5), kCbrt), c);
  double z3 = dmul(dmul(z, z), z);
  z = __fma_rn(dmul(z, __fma_rn(-a, z3, 1.0)), THIRD, z);   // Newton for a^(-1/3)
  double zz = dmul(z, z);
  double y = dmul(a, zz);
  double d;
  if (U10) {
    d2 y3 = mul_d2_d(mul_dd(y, y), y);
    d = __dadd_rn(__dsub_rn(y3.x, a), y3.y);
  } else {
    d = __fma_rn(dmul(y, y), y, -a);
  }
  y = __fma_rn(-d, dmul(zz, THIRD), y);                    // Newton for a^(1/3)
  y = dmul(y, pow2i(q - off));
  if (!fin) y = __dadd_rn(x, x);
  return canon(copysign_b(y, bx));
}
struct CbrtU10 { __device__ double operator()(double x) const { return cbrt_core<true>(x); } };
struct CbrtU35 { __device__ double operator()(double x) const { return cbrt_core<false>(x); } };

// ---------------- sinh, cosh, tanh ----------------
// sinh/cosh lanes split at |x| = 22 (DD formula or e^|x|/2), asinh/acosh at
// 2^500 (square root or not): the sorted-tile kernel keeps each warp on one
__device__ __forceinline__ int cls_22(double x) { return (bits(x) & ABS64) > 0x4036000000000000ull; }
__device__ __forceinline__ int cls_500(double x) { return (bits(x) & ABS64) > 0x5F30000000000000ull; }

struct SinhU10 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_22(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B711 ? from_bits(ab) : 0.0;
    double k;
    d2 s = expk_s(D2(ac, 0.0), k);
    double y;
    if (bits(ac) > 0x4036000000000000ull) {   // ac > 22
      d2 e = add_d_d2_fast(1.0, s);
      y = scale2(__dadd_rn(e.x, e.y), int_of(k) - 1);
    } else {
      d2 em = em1_join(s, k);
      d2 f = div_d2d2(em, add_d_d2(1.0, em));
      d2 h = add_d2d2(em, f);
      y = dmul(0.5, __dadd_rn(h.x, h.y));
    }
    if (ab < BM28) y = from_bits(ab);
    if (ab > B711) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(copysign_b(y, bx));
  }
};
struct CoshU10 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_22(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B711 ? from_bits(ab) : 0.0;
    double k;
    d2 s = expk_s(D2(ac, 0.0), k);
    d2 e = add_d_d2_fast(1.0, s);
    double y;
    if (bits(ac) > 0x4036000000000000ull) {   // ac > 22
      y = scale2(__dadd_rn(e.x, e.y), int_of(k) - 1);
    } else {
      d2 E = scale_d2(e, pow2i(int_of(k)));
      d2 h = add_d2d2_fast(E, rec_d2(E));
      y = dmul(0.5, __dadd_rn(h.x, h.y));
    }
    if (ab > B711) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(y);
  }
};
struct TanhU10 {
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B20 ? from_bits(ab) : 0.0;
    double k;
    d2 s = expk_s(D2(__dadd_rn(ac, ac), 0.0), k);
    d2 em = em1_join(s, k);
    d2 t = div_d2d2(em, add_d_d2(2.0, em));
    double y = __dadd_rn(t.x, t.y);
    if (ab < BM28) y = from_bits(ab);
    if (ab > B20) y = is_nan_b(bx) ? from_bits(QNAN64) : 1.0;
    return canon(copysign_b(y, bx));
  }
};
struct SinhU35 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_22(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B711 ? from_bits(ab) : 0.0;
    double k;
    double v = em1_u35(ac, k);
    double y;
    if (bits(ac) > 0x4036000000000000ull) {   // ac > 22
      y = scale2(__dadd_rn(1.0, v), int_of(k) - 1);
    } else {
      double p = pow2i(int_of(k));
      double em = __fma_rn(p, v, __dsub_rn(p, 1.0));
      y = dmul(0.5, __dadd_rn(em, dmul(em, __ddiv_rn(1.0, __dadd_rn(em, 1.0)))));
    }
    if (ab < BM28) y = from_bits(ab);
    if (ab > B711) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(copysign_b(y, bx));
  }
};
struct CoshU35 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_22(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B711 ? from_bits(ab) : 0.0;
    double k;
    double v = em1_u35(ac, k);
    double y;
    if (bits(ac) > 0x4036000000000000ull) {   // ac > 22
      y = scale2(__dadd_rn(1.0, v), int_of(k) - 1);
    } else {
      double E = dmul(__dadd_rn(1.0, v), pow2i(int_of(k)));
      y = dmul(0.5, __dadd_rn(E, __ddiv_rn(1.0, E)));
    }
    if (ab > B711) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(y);
  }
};
struct TanhU35 {
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= B20 ? from_bits(ab) : 0.0;
    double k;
    double v = em1_u35(__dadd_rn(ac, ac), k);
    double p = pow2i(int_of(k));
    double em = __fma_rn(p, v, __dsub_rn(p, 1.0));
    double y = dmul(em, __ddiv_rn(1.0, __dadd_rn(em, 2.0)));
    if (ab < BM28) y = from_bits(ab);
    if (ab > B20) y = is_nan_b(bx) ? from_bits(QNAN64) : 1.0;
    return canon(copysign_b(y, bx));
  }
};

// ---------------- asinh, acosh, atanh ----------------
struct AsinhU10 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_500(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= DMAX ? from_bits(ab) : 1.0;
    bool big = bits(ac) > 0x5F30000000000000ull;   // ac > 2^500
    d2 arg;
    if (big) {
      arg = D2(ac, 0.0);
    } else {
      d2 w = sqrt_d2(add_d2_d(mul_dd(ac, ac), 1.0));
      arg = add_d2_d(w, ac);
    }
    d2 r = log_dd(arg);
    if (big) r = add_d2d2(r, D2(L2A, L2B));
    double y = __dadd_rn(r.x, r.y);
    if (ab < BM28) y = from_bits(ab);
    if (ab > DMAX) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(copysign_b(y, bx));
  }
};
struct AcoshU10 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_500(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    bool inr = bx >= ONE && bx <= DMAX;              // 1 <= x < inf
    double xc = inr ? x : 1.0;
    bool big = bits(xc) > 0x5F30000000000000ull;   // xc > 2^500
    d2 arg;
    if (big) {
      arg = D2(xc, 0.0);
    } else {
      d2 d = mul_d2d2(add_dd(xc, -1.0), add_dd(xc, 1.0));
      arg = add_d2_d(sqrt_d2(d), xc);
    }
    d2 r = log_dd(arg);
    if (big) r = add_d2d2(r, D2(L2A, L2B));
    double y = __dadd_rn(r.x, r.y);
    if (bits(xc) == ONE) y = 0.0;
    if (!inr) y = bx == INF ? from_bits(INF) : from_bits(QNAN64);
    return canon(y);
  }
};
struct AtanhU10 {
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab < ONE ? from_bits(ab) : 0.5;
    d2 q = div_d2d2(add_dd(1.0, ac), add_dd(1.0, -ac));
    d2 r = log_dd(q);
    double y = dmul(0.5, __dadd_rn(r.x, r.y));
    if (ab < BM28) y = from_bits(ab);
    if (ab >= ONE) y = ab == ONE ? from_bits(INF) : from_bits(QNAN64);
    return canon(copysign_b(y, bx));
  }
};

// the 3.5-ULP forms: the same DD arguments, their logarithm in double with z
// corrected once (logm_u20) and e ln 2 added by one fma
struct AsinhU35 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_500(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab <= DMAX ? from_bits(ab) : 1.0;
    bool big = bits(ac) > 0x5F30000000000000ull;   // ac > 2^500
    d2 arg;
    if (big) {
      arg = D2(ac, 0.0);
    } else {
      d2 w = sqrt_d2(add_d2_d(mul_dd(ac, ac), 1.0));
      arg = add_d2_d(w, ac);
    }
    int e;
    double lm = logm_u20(arg, e);
    double y = __fma_rn(dbl_of(big ? e + 1 : e), L2A, lm);   // log(2 ac) above 2^500
    if (ab < BM28) y = from_bits(ab);
    if (ab > DMAX) y = is_nan_b(bx) ? from_bits(QNAN64) : from_bits(INF);
    return canon(copysign_b(y, bx));
  }
};
struct AcoshU35 {
  static constexpr int NCLS = 2;
  __device__ static int cls(double x) { return cls_500(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    bool inr = bx >= ONE && bx <= DMAX;              // 1 <= x < inf
    double xc = inr ? x : 1.0;
    bool big = bits(xc) > 0x5F30000000000000ull;   // xc > 2^500
    d2 arg;
    if (big) {
      arg = D2(xc, 0.0);
    } else {
      d2 d = mul_d2d2(add_dd(xc, -1.0), add_dd(xc, 1.0));
      arg = add_d2_d(sqrt_d2(d), xc);
    }
    int e;
    double lm = logm_u20(arg, e);
    double y = __fma_rn(dbl_of(big ? e + 1 : e), L2A, lm);
    if (bits(xc) == ONE) y = 0.0;
    if (!inr) y = bx == INF ? from_bits(INF) : from_bits(QNAN64);
    return canon(y);
  }
};
struct AtanhU35 {
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x), ab = bx & ABS64;
    double ac = ab < ONE ? from_bits(ab) : 0.5;
    d2 q = div_d2d2(add_dd(1.0, ac), add_dd(1.0, -ac));
    int e;
    double lm = logm_u20(q, e);
    double y = dmul(0.5, __fma_rn(dbl_of(e), L2A, lm));
    if (ab < BM28) y = from_bits(ab);
    if (ab >= ONE) y = ab == ONE ? from_bits(INF) : from_bits(QNAN64);
    return canon(copysign_b(y, bx));
  }
};


// ---------------- erf, erfc ----------------
// erf: |x| < 1: x (C0 + T (C1 + T (c2 + t P(t)))), T = x^2 exact, the three
// outer levels in DD; 1 <= |x| < 6: 1 - erfc(|x|) in DD; +-1 beyond.
// erfc: |x| < 1: 1 -+ erf(|x|) in DD; 1 <= |x| <= 27.5: F(|x|) e^(-x^2) with
// F = erfc e^(x^2) a polynomial about the midpoint of [1,2), [2,4), [4,8)
// (two leading terms in DD) or G(1/x^2) / (sqrt(pi) x) from 8 on; e^(-x^2)
// from the DD exp core on the exact DD x^2; 2^k applied by two
// multiplications (one rounding for subnormal results); erfc(-x) = 2 - erfc(x).
// The tile sort groups lanes by interval so that each warp reads one row of
// the coefficient tables.  u35 erf: the same pieces in double; u35 erfc runs
// the u10 algorithm.
constexpr double RSQPIH = 0x1.20dd750429b6dp-1, RSQPIL = 0x1.1ae3a914f6e1fp-57;   // 1/sqrt(pi)
static __constant__ double kErfH[4] = {0x1.20dd750429b6dp+0, 0x1.18308016146fep-56, -0x1.812746b0379e6p-2, 0x1.dd80e959672c6p-58};
static __constant__ double kErfP[11] = {
    0x1.ce2f21a042b20p-4, -0x1.b82ce31284967p-6, 0x1.565bcd0daf845p-8, -0x1.c02db3d8c8f93p-11,
    0x1.f9a3219c76949p-14, -0x1.f4d1ded722b03p-17, 0x1.b9deec50ab26ap-20, -0x1.5f1d06eacf4c6p-23,
    0x1.f7a1f36ad5781p-27, -0x1.3863e3c35d413p-30, 0x1.0566538cb8283p-34};
static __constant__ double kErfcFH[3][4] = {
    {0x1.494daffa2ad68p-2, 0x1.39bdf0f0798c4p-56, -0x1.4f1988444caf7p-3, 0x1.24ac537655c12p-57},
    {0x1.6e9827d229d2dp-3, -0x1.90756fe6b9db3p-58, -0x1.bd6ae4d14b16fp-5, 0x1.8d8b238907b15p-61},
    {0x1.7c0348489d721p-4, 0x1.ca79ab435b660p-58, -0x1.ed7f66d9d09fep-7, 0x1.3b520acfa96f3p-62}};
static __constant__ double kErfcFP[3][22] = {
  {
    0x1.37ea271bc54bdp-4, -0x1.0dc51d2941e6dp-5, 0x1.b65944f34f7adp-7, -0x1.513ed7600d1c0p-8,
    0x1.ee705e736464dp-10, -0x1.5b0abfe65a32dp-11, 0x1.d4509d0d417b9p-13, -0x1.30c0ec743bcedp-14,
    0x1.7f997923557c4p-16, -0x1.d4157188ae920p-18, 0x1.156c936a3105dp-19, -0x1.4004eff6f7f58p-21,
    0x1.67cf5f0988c05p-23, -0x1.8adc1a9fe6189p-25, 0x1.a779871f4a7bdp-27, -0x1.bc5770d3295a2p-29,
    0x1.c8a6eada5b280p-31, -0x1.cbfeb0383b565p-33, 0x1.c520022695974p-35, -0x1.b81dd79ebf9adp-37,
    0x1.c82b760607022p-39, -0x1.a70fd6017ce87p-41},
  {
    0x1.043fe1a98c0cdp-6, -0x1.259061ba85692p-8, 0x1.409cc2ed3fefbp-10, -0x1.53dec9d089553p-12,
    0x1.5e739304850bcp-14, -0x1.6025103c1981bp-16, 0x1.595f1b5dbff18p-18, -0x1.4b14628647c09p-20,
    0x1.369904b947a56p-22, -0x1.1d791455a0f11p-24, 0x1.01508df8e0a1fp-26, -0x1.c752068f0a96ep-29,
    0x1.8bbf3f6db12c5p-31, -0x1.522804d7a7020p-33, 0x1.1c3dc4fa8a305p-35, -0x1.d66d6369f7643p-38,
    0x1.8003b981c62cdp-40, -0x1.3453718d4c0bfp-42, 0x1.dbc8fa69f1588p-45, -0x1.7551e98792b95p-47,
    0x1.6ca3dddd58940p-49, -0x1.10f3c57b6b0d7p-51},
  {
    0x1.3c7764a81f462p-9, -0x1.9106a7cd79e3bp-12, 0x1.f64cd9c07b5c5p-15, -0x1.370d0641775e4p-17,
    0x1.7d0e03edb73e5p-20, -0x1.cde4cecce654ep-23, 0x1.1513469d8602cp-25, -0x1.491bb0ca940c5p-28,
    0x1.83201ae0eb1dcp-31, -0x1.c312ca4fcf13cp-34, 0x1.045ff3e648ff3p-36, -0x1.29e5d7aaf7613p-39,
    0x1.51dbcb9512727p-42, -0x1.7be13c8006386p-45, 0x1.a72a1d41d3c2ap-48, -0x1.d40a279e38d1dp-51,
    0x1.040a46c482170p-53, -0x1.1a97bd1e37a50p-56, 0x1.0dfc0cce80407p-59, -0x1.24502b98063a1p-62,
    0x1.0709dd4f990c4p-64, -0x1.11b59748cdbf2p-67}};
static __constant__ double kErfcGH[4] = {0x1.0000000000000p+0, -0x1.38b4a1f7dc331p-66, -0x1.ffffffffffffbp-2, -0x1.449ed132ba430p-56};
static __constant__ double kErfcGP[9] = {
    0x1.7ffffffffe83fp-1, -0x1.dffffffd0f32bp+0, 0x1.a3fffe80c9ac6p+2, -0x1.d87f8dc75c4bdp+4,
    0x1.44cd52e365bc6p+7, -0x1.0749c46c91cccp+10, 0x1.e1ba8d8295a72p+12, -0x1.b7be9d06eea96p+15,
    0x1.142dd87ba7a2cp+18};

__device__ __forceinline__ d2 neg_d2(d2 a) { return D2(-a.x, -a.y); }
// erf(a)/a as a DD, 0 <= a < 1
__device__ __forceinline__ d2 erf_s(double a) {
  d2 T = mul_dd(a, a);
  double p = poly_p<10>(T.x, kErfP + 1);
  d2 in = add_dd(kErfP[0], dmul(T.x, p));
  in = add_d2d2(D2(kErfH[2], kErfH[3]), mul_d2d2(T, in));
  return add_d2d2(D2(kErfH[0], kErfH[1]), mul_d2d2(T, in));
}
// interval bounds as bit patterns: a >= 0 (or +NaN), so the order of the
// bits is the order of the values
constexpr uint64_t BE1 = 0x3FF0000000000000ull, BE2 = 0x4000000000000000ull, BE4 = 0x4010000000000000ull;
constexpr uint64_t BE6 = 0x4018000000000000ull, BE8 = 0x4020000000000000ull, BE275 = 0x403B800000000000ull;
__device__ __forceinline__ int erfc_iv(double a) { return bits(a) < BE2 ? 0 : (bits(a) < BE4 ? 1 : 2); }
// F(a) = erfc(a) e^(a^2) as a DD, 1 <= a <= 27.5
__device__ __forceinline__ d2 erfc_F(double a) {
  if (bits(a) < BE8) {
    int i = erfc_iv(a);
    double u = __dsub_rn(a, i == 0 ? 1.5 : (i == 1 ? 3.0 : 6.0));
    double p = poly_p<22>(u, kErfcFP[i]);
    d2 in = add_d2_d(D2(kErfcFH[i][2], kErfcFH[i][3]), dmul(u, p));
    return add_d2d2(D2(kErfcFH[i][0], kErfcFH[i][1]), mul_d2_d(in, u));
  }
  double w = __ddiv_rn(1.0, dmul(a, a));
  double p = poly_p<9>(w, kErfcGP);
  d2 in = add_d2_d(D2(kErfcGH[2], kErfcGH[3]), dmul(w, p));
  d2 g = add_d2d2(D2(kErfcGH[0], kErfcGH[1]), mul_d2_d(in, w));
  return div_d2d2(mul_d2d2(g, D2(RSQPIH, RSQPIL)), D2(a, 0.0));
}
// erfc(a) = c 2^k, 1 <= a <= 27.5
__device__ __forceinline__ d2 erfc_core(double a, double &k) {
  d2 Y = mul_dd(a, a);
  d2 s = expk_s(D2(-Y.x, -Y.y), k);
  return mul_d2d2(erfc_F(a), add_d_d2_fast(1.0, s));
}
// y 2^k by two multiplications with normal powers of two (one rounding)
__device__ __forceinline__ double scale2_two(double y, int k) {
  int k1 = k / 2, k2 = k - k1;
  return dmul(dmul(y, pow2i(k1)), pow2i(k2));
}

struct ErfU10 {
  static constexpr int NCLS = 5;
  static constexpr int SORT_EPT = 8;    // 2048-element tiles
  __device__ static int cls(double x) {
    uint64_t a = bits(x) & ABS64;
    return a < BE1 ? 0 : (a < BE2 ? 1 : (a < BE4 ? 2 : (a < BE6 ? 3 : 4)));
  }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    double a = from_bits(bx & ABS64);
    double y;
    if (bits(a) < BE1) {
      d2 e = mul_d2_d(erf_s(a), a);
      y = __dadd_rn(e.x, e.y);
    } else if (bits(a) < BE6) {
      double k;
      d2 c = erfc_core(a, k);
      c = scale_d2(c, pow2i(int_of(k)));
      d2 r = add_d_d2(1.0, neg_d2(c));
      y = __dadd_rn(r.x, r.y);
    } else {
      y = 1.0;
    }
    if (is_nan_b(bx)) y = from_bits(QNAN64);
    return canon(copysign_b(y, bx));
  }
};
struct ErfcU10 {
  static constexpr int NCLS = 6;
  static constexpr int SORT_EPT = 8;    // 2048-element tiles
  __device__ static int cls(double x) {
    uint64_t a = bits(x) & ABS64;
    return a < BE1 ? 0 : (a < BE2 ? 1 : (a < BE4 ? 2 : (a < BE8 ? 3 : (a <= BE275 ? 4 : 5))));
  }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    double a = from_bits(bx & ABS64);
    double y;
    if (bits(a) < BE1) {
      d2 e = mul_d2_d(erf_s(a), a);
      if (gt_0(x)) e = neg_d2(e);
      d2 r = add_d_d2(1.0, e);
      y = __dadd_rn(r.x, r.y);
    } else if (bits(a) <= BE275) {
      double k;
      d2 c = erfc_core(a, k);
      if (gt_0(x)) {
        y = scale2_two(__dadd_rn(c.x, c.y), int_of(k));
      } else if (bits(a) < BE8) {
        c = scale_d2(c, pow2i(int_of(k)));
        d2 r = add_d_d2(2.0, neg_d2(c));
        y = __dadd_rn(r.x, r.y);
      } else {
        y = 2.0;
      }
    } else {
      y = gt_0(x) ? 0.0 : 2.0;
    }
    if (is_nan_b(bx)) y = from_bits(QNAN64);
    return canon(y);
  }
};
struct ErfU35 {
  static constexpr int NCLS = 5;
  static constexpr int SORT_EPT = 8;    // 2048-element tiles
  __device__ static int cls(double x) { return ErfU10::cls(x); }
  __device__ double operator()(double x) const {
    uint64_t bx = bits(x);
    double a = from_bits(bx & ABS64);
    double y;
    if (bits(a) < BE1) {
      double t = dmul(a, a);
      y = dmul(a, __fma_rn(t, __fma_rn(t, poly(t, kErfP), kErfH[2]), kErfH[0]));
    } else if (bits(a) < BE6) {
      int i = erfc_iv(a);
      double u = __dsub_rn(a, i == 0 ? 1.5 : (i == 1 ? 3.0 : 6.0));
      double F = __fma_rn(u, __fma_rn(u, poly_p<22>(u, kErfcFP[i]), kErfcFH[i][2]), kErfcFH[i][0]);
      d2 Y = mul_dd(a, a);
      double k = drint(dmul(-Y.x, R_LN2));
      double r = __dsub_rn(__fma_rn(k, -L2B, __fma_rn(k, -L2A, -Y.x)), Y.y);
      double E = dmul(__dadd_rn(1.0, em1_r_u35(r)), pow2i(int_of(k)));
      y = __fma_rn(-F, E, 1.0);
    } else {
      y = 1.0;
    }
    if (is_nan_b(bx)) y = from_bits(QNAN64);
    return canon(copysign_b(y, bx));
  }
};

}  // namespace derived64
}  // namespace sleefcu

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define UNARY64(NAME, F)                                                                    \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_unary64<derived64::F>("sleefcu_" #NAME, x, out, n, s);                    \
  }
#define UNARY64_MASKED(NAME, F)                                                     \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<derived64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
#define SORTED64(NAME, F)                                                                   \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_sorted64<derived64::F>("sleefcu_" #NAME, x, out, n, s);                   \
  }
#define SORTED64_MASKED(NAME, F)                                                    \
  extern "C" sleefcu_status sleefcu_##NAME##_masked(const double *x, const uint8_t *mask,  \
                                                    double *out, size_t n, sleefcu_stream s) { \
    return launch_masked64<derived64::F>("sleefcu_" #NAME "_masked", x, mask, out, n, s);         \
  }
UNARY64(exp2_u10_f64, Exp2U10)
UNARY64_MASKED(exp2_u10_f64, Exp2U10)
UNARY64(exp2_u35_f64, Exp2U35)
UNARY64_MASKED(exp2_u35_f64, Exp2U35)
UNARY64(exp10_u10_f64, Exp10U10)
UNARY64_MASKED(exp10_u10_f64, Exp10U10)
UNARY64(exp10_u35_f64, Exp10U35)
UNARY64_MASKED(exp10_u35_f64, Exp10U35)
UNARY64(expm1_u10_f64, Expm1U10)
UNARY64_MASKED(expm1_u10_f64, Expm1U10)
UNARY64(expm1_u35_f64, Expm1U35)
UNARY64_MASKED(expm1_u35_f64, Expm1U35)
UNARY64(log2_u10_f64, Log2U10)
UNARY64_MASKED(log2_u10_f64, Log2U10)
UNARY64(log2_u35_f64, Log2U35)
UNARY64_MASKED(log2_u35_f64, Log2U35)
UNARY64(log10_u10_f64, Log10U10)
UNARY64_MASKED(log10_u10_f64, Log10U10)
UNARY64(log10_u35_f64, Log10U35)
UNARY64_MASKED(log10_u35_f64, Log10U35)
UNARY64(log1p_u10_f64, Log1pU10)
UNARY64_MASKED(log1p_u10_f64, Log1pU10)
UNARY64(log1p_u35_f64, Log1pU35)
UNARY64_MASKED(log1p_u35_f64, Log1pU35)
UNARY64(cbrt_u10_f64, CbrtU10)
UNARY64_MASKED(cbrt_u10_f64, CbrtU10)
UNARY64(cbrt_u35_f64, CbrtU35)
UNARY64_MASKED(cbrt_u35_f64, CbrtU35)
SORTED64(sinh_u10_f64, SinhU10)
SORTED64_MASKED(sinh_u10_f64, SinhU10)
SORTED64(sinh_u35_f64, SinhU35)
SORTED64_MASKED(sinh_u35_f64, SinhU35)
SORTED64(cosh_u10_f64, CoshU10)
SORTED64_MASKED(cosh_u10_f64, CoshU10)
SORTED64(cosh_u35_f64, CoshU35)
SORTED64_MASKED(cosh_u35_f64, CoshU35)
UNARY64(tanh_u10_f64, TanhU10)
UNARY64_MASKED(tanh_u10_f64, TanhU10)
UNARY64(tanh_u35_f64, TanhU35)
UNARY64_MASKED(tanh_u35_f64, TanhU35)
SORTED64(asinh_u10_f64, AsinhU10)
SORTED64_MASKED(asinh_u10_f64, AsinhU10)
SORTED64(asinh_u35_f64, AsinhU35)
SORTED64_MASKED(asinh_u35_f64, AsinhU35)
SORTED64(acosh_u10_f64, AcoshU10)
SORTED64_MASKED(acosh_u10_f64, AcoshU10)
SORTED64(acosh_u35_f64, AcoshU35)
SORTED64_MASKED(acosh_u35_f64, AcoshU35)
SORTED64(erf_u10_f64, ErfU10)
SORTED64_MASKED(erf_u10_f64, ErfU10)
SORTED64(erf_u35_f64, ErfU35)
SORTED64_MASKED(erf_u35_f64, ErfU35)
SORTED64(erfc_u10_f64, ErfcU10)
SORTED64_MASKED(erfc_u10_f64, ErfcU10)
SORTED64(erfc_u35_f64, ErfcU10)
SORTED64_MASKED(erfc_u35_f64, ErfcU10)
UNARY64(atanh_u10_f64, AtanhU10)
UNARY64_MASKED(atanh_u10_f64, AtanhU10)
UNARY64(atanh_u35_f64, AtanhU35)
UNARY64_MASKED(atanh_u35_f64, AtanhU35)
#undef UNARY64
#undef UNARY64_MASKED
#undef SORTED64
#undef SORTED64_MASKED
#endif  // SLEEFCU_FUNCTORS_ONLY
