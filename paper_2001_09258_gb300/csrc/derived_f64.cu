// FP64 functions built on the exp/log cores (u10 and u35) for sm_103a:
// exp2, exp10, expm1, log2, log10, log1p, cbrt, sinh, cosh, tanh, asinh,
// acosh, atanh.  The paper lists them in the library without giving their
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
  return __fma_rn(__dmul_rn(t, t), poly(t, kExpm1U35), t);
}
// 2^k s + (2^k - 1) as a DD (k <= 1000), 2^k - 1 formed exactly by TwoSum
__device__ __forceinline__ d2 em1_join(d2 s, double k) {
  double p = pow2i(int_of(k));
  return add_d2d2(add_dd(p, -1.0), scale_d2(s, p));
}
// k and e^r - 1 in double for the u35 forms
__device__ __forceinline__ double em1_u35(double xc, double &k) {
  k = rint(__dmul_rn(xc, R_LN2));
  double r = __fma_rn(k, -L2B, __fma_rn(k, -L2A, xc));
  return em1_r_u35(r);
}
// log of a DD a > 0 as a DD
__device__ __forceinline__ d2 log_dd(d2 a) {
  int e;
  d2 lm = logm_u10(a, e);
  double ed = dbl_of(e);
  return add_d2d2(D2(__dmul_rn(ed, L2H), __dmul_rn(ed, L2L)), lm);
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
    double k = rint(xc);
    d2 t = mul_d2_d(D2(L2A, L2B), __dsub_rn(xc, k));
    return exp_out(b, inr, exp_tail_u10(t.x, t.y, int_of(k)));
  }
};
struct Exp2U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B1100;
    double xc = inr ? x : 0.0;
    double k = rint(xc);
    double t = __dmul_rn(__dsub_rn(xc, k), L2A);
    return exp_out(b, inr, scale2(__dadd_rn(1.0, em1_r_u35(t)), int_of(k)));
  }
};
struct Exp10U10 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    bool inr = (b & ABS64) <= B350;
    double xc = inr ? x : 0.0;
    double k = rint(__dmul_rn(xc, LOG2_10));
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
    double k = rint(__dmul_rn(xc, LOG2_10));
    double r = __fma_rn(k, -L10B, __fma_rn(k, -L10A, xc));
    return exp_out(b, inr, scale2(__dadd_rn(1.0, em1_r_u35(__dmul_rn(r, LN10H))), int_of(k)));
  }
};

// ---------------- expm1 ----------------
__device__ __forceinline__ double expm1_out(double x, double y) {
  bool inr = x > -40.0 && x < 710.0;
  if (x == 0.0) y = x;
  if (!inr) y = x >= 710.0 ? from_bits(INF) : (x <= -40.0 ? -1.0 : from_bits(QNAN64));
  return canon(y);
}
struct Expm1U10 {
  __device__ double operator()(double x) const {
    double xc = (x > -40.0 && x < 710.0) ? x : 0.0;
    double k;
    d2 s = expk_s(D2(xc, 0.0), k);
    double y;
    if (k > 1000.0) {
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
    double xc = (x > -40.0 && x < 710.0) ? x : 0.0;
    double k;
    double v = em1_u35(xc, k);
    double y;
    if (k > 1000.0) {
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
    d2 r = add_d2d2(D2(__dmul_rn(ed, LG2H), __dmul_rn(ed, LG2L)), p);
    return log_out(b, __dadd_rn(r.x, r.y));
  }
};
struct Log10U35 {
  __device__ double operator()(double x) const {
    uint64_t b = bits(x);
    int e;
    d2 lm = logm_u10(D2(log_arg(b), 0.0), e);
    return log_out(b, __fma_rn(dbl_of(e), L10A, __dmul_rn(__dadd_rn(lm.x, lm.y), RL10H)));
  }
};
__device__ __forceinline__ double log1p_out(double x, double y) {
  if (x == -1.0) return from_bits(0xFFF0000000000000ull);
  if (x < -1.0 || x != x) return from_bits(QNAN64);
  if (bits(x) == INF) return from_bits(INF);
  if (x == 0.0) return x;
  return canon(y);
}
__device__ __forceinline__ double log1p_arg(double x) {
  return (x > -1.0 && (bits(x) & ABS64) <= DMAX) ? x : 0.0;
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
  if (a0 < 0x1p-1022) { a0 = __dmul_rn(a0, 0x1p54); off = 18; }
  uint64_t b0 = bits(a0);
  int e = (int)(b0 >> 52) - 1023;
  int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  int i = e - 3 * q;
  double m = from_bits((b0 & 0x000FFFFFFFFFFFFFull) | ONE);     // [1, 2)
  double a = __dmul_rn(m, pow2i(i));                             // [1, 8)
  double c = i == 0 ? 1.0 : (i == 1 ? CBRT_C1 : CBRT_C2);
  double z = __dmul_rn(poly(__dsub_rn(m, 1.5), kCbrt), c);
  double z3 = __dmul_rn(__dmul_rn(z, z), z);
  z = __fma_rn(__dmul_rn(z, __fma_rn(-a, z3, 1.0)), THIRD, z);   // Newton for a^(-1/3)
  double zz = __dmul_rn(z, z);
  double y = __dmul_rn(a, zz);
  double d;
  if (U10) {
    d2 y3 = mul_d2_d(mul_dd(y, y), y);
    d = __dadd_rn(__dsub_rn(y3.x, a), y3.y);
  } else {
    d = __fma_rn(__dmul_rn(y, y), y, -a);
  }
  y = __fma_rn(-d, __dmul_rn(zz, THIRD), y);                    // Newton for a^(1/3)
  y = __dmul_rn(y, pow2i(q - off));
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
    if (ac > 22.0) {
      d2 e = add_d_d2_fast(1.0, s);
      y = scale2(__dadd_rn(e.x, e.y), int_of(k) - 1);
    } else {
      d2 em = em1_join(s, k);
      d2 f = div_d2d2(em, add_d_d2(1.0, em));
      d2 h = add_d2d2(em, f);
      y = __dmul_rn(0.5, __dadd_rn(h.x, h.y));
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
    if (ac > 22.0) {
      y = scale2(__dadd_rn(e.x, e.y), int_of(k) - 1);
    } else {
      d2 E = scale_d2(e, pow2i(int_of(k)));
      d2 h = add_d2d2_fast(E, rec_d2(E));
      y = __dmul_rn(0.5, __dadd_rn(h.x, h.y));
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
    if (ac > 22.0) {
      y = scale2(__dadd_rn(1.0, v), int_of(k) - 1);
    } else {
      double p = pow2i(int_of(k));
      double em = __fma_rn(p, v, __dsub_rn(p, 1.0));
      y = __dmul_rn(0.5, __dadd_rn(em, __ddiv_rn(em, __dadd_rn(em, 1.0))));
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
    if (ac > 22.0) {
      y = scale2(__dadd_rn(1.0, v), int_of(k) - 1);
    } else {
      double E = __dmul_rn(__dadd_rn(1.0, v), pow2i(int_of(k)));
      y = __dmul_rn(0.5, __dadd_rn(E, __ddiv_rn(1.0, E)));
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
    double y = __ddiv_rn(em, __dadd_rn(em, 2.0));
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
    bool big = ac > 0x1p500;
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
    bool inr = x >= 1.0 && bx <= DMAX;
    double xc = inr ? x : 1.0;
    bool big = xc > 0x1p500;
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
    if (xc == 1.0) y = 0.0;
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
    double y = __dmul_rn(0.5, __dadd_rn(r.x, r.y));
    if (ab < BM28) y = from_bits(ab);
    if (ab >= ONE) y = ab == ONE ? from_bits(INF) : from_bits(QNAN64);
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
#define SORTED64(NAME, F)                                                                   \
  extern "C" sleefcu_status sleefcu_##NAME(const double *x, double *out, size_t n,          \
                                           sleefcu_stream s) {                              \
    return launch_sorted64<derived64::F>("sleefcu_" #NAME, x, out, n, s);                   \
  }
UNARY64(exp2_u10_f64, Exp2U10)
UNARY64(exp2_u35_f64, Exp2U35)
UNARY64(exp10_u10_f64, Exp10U10)
UNARY64(exp10_u35_f64, Exp10U35)
UNARY64(expm1_u10_f64, Expm1U10)
UNARY64(expm1_u35_f64, Expm1U35)
UNARY64(log2_u10_f64, Log2U10)
UNARY64(log2_u35_f64, Log2U35)
UNARY64(log10_u10_f64, Log10U10)
UNARY64(log10_u35_f64, Log10U35)
UNARY64(log1p_u10_f64, Log1pU10)
UNARY64(log1p_u35_f64, Log1pU35)
UNARY64(cbrt_u10_f64, CbrtU10)
UNARY64(cbrt_u35_f64, CbrtU35)
SORTED64(sinh_u10_f64, SinhU10)
SORTED64(sinh_u35_f64, SinhU35)
SORTED64(cosh_u10_f64, CoshU10)
SORTED64(cosh_u35_f64, CoshU35)
UNARY64(tanh_u10_f64, TanhU10)
UNARY64(tanh_u35_f64, TanhU35)
SORTED64(asinh_u10_f64, AsinhU10)
SORTED64(asinh_u35_f64, AsinhU10)
SORTED64(acosh_u10_f64, AcoshU10)
SORTED64(acosh_u35_f64, AcoshU10)
UNARY64(atanh_u10_f64, AtanhU10)
UNARY64(atanh_u35_f64, AtanhU10)
#undef UNARY64
#undef SORTED64
#endif  // SLEEFCU_FUNCTORS_ONLY
