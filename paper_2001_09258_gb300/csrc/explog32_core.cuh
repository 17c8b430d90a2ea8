// FP32 exp/log cores and the exp, log, log1p, tanh, erf functors shared by
// the FP32 entry points, the 16-bit forms and the functions built on them.
#pragma once
#include "sleefcu_common.cuh"

namespace sleefcu {
namespace explog32 {

constexpr float R_LN2F = 0x1.715476p0f, L2AF = 0x1.62e430p-1f, L2BF = -0x1.05c610p-29f;
constexpr float L2HF = 0x1.62e400p-1f, L2LF = 0x1.7f7d1cp-20f;
constexpr uint32_t B104 = 0x42d00000u, B1 = 0x3f800000u, B395 = 0x407ccccdu, B91 = 0x4111999au;
constexpr uint32_t FMAX = 0x7F7FFFFFu, INF = 0x7F800000u;
constexpr float ERF_C = 2.475f;

static __constant__ float kExpU10[6] = {
  0x1.0000000000000p-1f, 0x1.55553c0000000p-3f, 0x1.5554f20000000p-5f, 0x1.1137480000000p-7f,
  0x1.6d41420000000p-10f, 0x1.6b42520000000p-13f};
static __constant__ float kExpU35[5] = {
  0x1.fffffc0000000p-2f, 0x1.55548c0000000p-3f, 0x1.5558580000000p-5f, 0x1.123da60000000p-7f,
  0x1.6ac36c0000000p-10f};
static __constant__ float kLogU10[4] = {
  0x1.5555540000000p-4f, 0x1.999c0c0000000p-7f, 0x1.23e0440000000p-9f, 0x1.ee9f240000000p-12f};
static __constant__ float kLogU35[3] = {
  0x1.5555b40000000p-4f, 0x1.992a9a0000000p-7f, 0x1.36eeb60000000p-9f};
static __constant__ float kExpm1[5] = {
  0x1.5555540000000p-3f, 0x1.5554e40000000p-5f, 0x1.1112de0000000p-7f, 0x1.6d520e0000000p-10f,
  0x1.9e7a5c0000000p-13f};
constexpr float ERFA_C0H = 0x1.20dd760000000p+0f, ERFA_C0L = -0x1.f7ff040000000p-25f;
static __constant__ float kErfA[7] = {
  -0x1.8127460000000p-2f, 0x1.ce2eea0000000p-4f, -0x1.b8269c0000000p-6f, 0x1.5604160000000p-8f,
  -0x1.bafc920000000p-11f, 0x1.cd9a840000000p-14f, -0x1.2acec00000000p-17f};
constexpr float ERFB_C0H = -0x1.8c474e0000000p+0f, ERFB_C0L = 0x1.b8d2c00000000p-28f;
static __constant__ float kErfB[11] = {
  -0x1.6c09ea0000000p-2f, 0x1.d25c580000000p-5f, -0x1.6afadc0000000p-7f, 0x1.22d4da0000000p-9f,
  -0x1.c5b2a40000000p-12f, 0x1.4c37b80000000p-14f, -0x1.b6e1140000000p-17f, 0x1.f87af20000000p-20f,
  -0x1.78eb0c0000000p-23f, -0x1.83d9360000000p-25f, 0x1.51170e0000000p-26f};

__device__ __forceinline__ int int_off(float k) {      // integer-valued float, |k| < 2^24
  uint32_t b = fbits(k);
  int e = (int)((b >> 23) & 0xFF) - 127;
  uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
  int v = e < 0 ? 0 : (int)(m >> (23 - e));
  return (b >> 31) ? -v : v;
}
__device__ __forceinline__ float fl_of(int v) { return __int2float_rn(v); }   // exact for |v| < 2^24
__device__ __forceinline__ float pow2f(int k) { return from_fbits((uint32_t)(k + 127) << 23); }
// y * 2^k (y in [0.5, 2)): exponent-field add when the result is normal,
// else two multiplications that round once
__device__ __forceinline__ float scale2f(float y, int k) {
  if (k >= -125 && k <= 127) return from_fbits(fbits(y) + ((uint32_t)k << 23));
  int k1 = k / 2, k2 = k - k1;
  return __fmul_rn(__fmul_rn(y, pow2f(k1)), pow2f(k2));
}
__device__ __forceinline__ float exp_sel(uint32_t b, float y) {
  if (!((b & ABS32) <= B104))
    y = (b & ABS32) > INF ? from_fbits(QNAN32) : ((b >> 31) ? 0.0f : from_fbits(INF));
  return canonf(y);
}

struct ExpU10 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x);
    float xc = (b & ABS32) <= B104 ? x : 0.0f;
    float k = rintf(__fmul_rn(xc, R_LN2F));
    float h = __fmaf_rn(k, -L2AF, xc);
    float r = __fmaf_rn(k, -L2BF, h);
    float rl = __fmaf_rn(k, -L2BF, __fsub_rn(h, r));
    float w = __fmaf_rn(__fmul_rn(r, r), polyf(r, kExpU10), rl);
    f2 o = add_ff_fast(1.0f, r);
    return exp_sel(b, scale2f(__fadd_rn(o.x, __fadd_rn(o.y, w)), int_off(k)));
  }
};
struct ExpU35 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x);
    float xc = (b & ABS32) <= B104 ? x : 0.0f;
    float k = rintf(__fmul_rn(xc, R_LN2F));
    float r = __fmaf_rn(k, -L2BF, __fmaf_rn(k, -L2AF, xc));
    float v = __fmaf_rn(__fmul_rn(r, r), polyf(r, kExpU35), r);
    return exp_sel(b, scale2f(__fadd_rn(1.0f, v), int_off(k)));
  }
};

// a: bits of a finite positive float; m in [0.75, 1.5), a = m 2^e
__device__ __forceinline__ float log_reduce(uint32_t a, int &e) {
  int off = 0;
  if (a < 0x00800000u) {
    a = fbits(__fmul_rn(from_fbits(a), 0x1p32f));
    off = 32;
  }
  int ex = (int)(a >> 23) - 127;
  uint32_t mb = (a & 0x7FFFFFu) | 0x3F800000u;
  if (mb & 0x00400000u) { mb -= 0x00800000u; ex++; }
  e = ex - off;
  return from_fbits(mb);
}
__device__ __forceinline__ f2 log_core_u10(float m, float ml, int e) {
  f2 num = scale_f2(add_ff(__fsub_rn(m, 1.0f), ml), 2.0f);
  f2 den = add_f_f2(1.0f, F2(m, ml));
  f2 z = div_f2f2(num, den);
  float t = __fmul_rn(z.x, z.x);
  float corr = __fmul_rn(__fmul_rn(z.x, t), polyf(t, kLogU10));
  float ed = fl_of(e);
  f2 r = add_f2f2_fast(F2(__fmul_rn(ed, L2HF), __fmul_rn(ed, L2LF)), z);
  return add_f2_f_fast(r, corr);
}
__device__ __forceinline__ float log_special(uint32_t b, float y) {
  if ((b & ABS32) == 0) return from_fbits(0xFF800000u);
  if ((b >> 31) || (b & ABS32) > INF) return from_fbits(QNAN32);
  if (b == INF) return from_fbits(INF);
  return y;
}
struct LogU10 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x);
    uint32_t a = (b - 1u) < FMAX ? b : B1;
    int e;
    float m = log_reduce(a, e);
    f2 r = log_core_u10(m, 0.0f, e);
    return canonf(log_special(b, __fadd_rn(r.x, r.y)));
  }
};
struct LogU35 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x);
    uint32_t a = (b - 1u) < FMAX ? b : B1;
    int e;
    float m = log_reduce(a, e);
    float z = __fdiv_rn(__fmul_rn(2.0f, __fsub_rn(m, 1.0f)), __fadd_rn(1.0f, m));
    float t = __fmul_rn(z, z);
    float lm = __fmaf_rn(__fmul_rn(z, t), polyf(t, kLogU35), z);
    return canonf(log_special(b, __fmaf_rn(fl_of(e), L2AF, lm)));
  }
};

__device__ __forceinline__ float log1p_special(float x, float y) {
  uint32_t b = fbits(x), ab = b & ABS32;
  if (b == 0xBF800000u) return from_fbits(0xFF800000u);            // -1 -> -inf
  if (ab > INF || ((b >> 31) && ab > B1)) return from_fbits(QNAN32);
  if (b == INF) return from_fbits(INF);
  if (ab == 0) return x;
  return y;
}
__device__ __forceinline__ bool log1p_ok(float x) {   // -1 < x <= FLT_MAX
  uint32_t b = fbits(x), ab = b & ABS32;
  return (b >> 31) ? ab < B1 : ab <= FMAX;
}
__device__ __forceinline__ float ldexp_small(float v, int e) {   // v * 2^-e, exact for normal results
  int e1 = e / 2;
  return __fmul_rn(__fmul_rn(v, pow2f(-e1)), pow2f(e1 - e));
}
struct Log1pU10 {
  __device__ float operator()(float x) const {
    float xc = log1p_ok(x) ? x : 0.0f;
    f2 s = add_ff(1.0f, xc);
    int e;
    float m = log_reduce(fbits(s.x), e);
    float ml = ldexp_small(s.y, e);
    f2 r = log_core_u10(m, ml, e);
    return canonf(log1p_special(x, __fadd_rn(r.x, r.y)));
  }
};
struct Log1pU35 {
  __device__ float operator()(float x) const {
    float xc = log1p_ok(x) ? x : 0.0f;
    f2 s = add_ff(1.0f, xc);
    int e;
    float m = log_reduce(fbits(s.x), e);
    float ml = ldexp_small(s.y, e);
    float z = __fdiv_rn(__fmul_rn(2.0f, __fadd_rn(__fsub_rn(m, 1.0f), ml)),
                        __fadd_rn(__fadd_rn(1.0f, m), ml));
    float t = __fmul_rn(z, z);
    float lm = __fmaf_rn(__fmul_rn(z, t), polyf(t, kLogU35), z);
    return canonf(log1p_special(x, __fmaf_rn(fl_of(e), L2AF, lm)));
  }
};

// expm1(a) in FF for 0 <= a <= 18.2
__device__ __forceinline__ f2 expm1_ff(float a) {
  float k = rintf(__fmul_rn(a, R_LN2F));
  float h = __fmaf_rn(k, -L2AF, a);
  float r = __fmaf_rn(k, -L2BF, h);
  float rl = __fmaf_rn(k, -L2BF, __fsub_rn(h, r));
  f2 rr = F2(r, rl);
  f2 q = scale_f2(sqr_f2(rr), 0.5f);
  float v = __fmul_rn(__fmul_rn(__fmul_rn(r, r), r), polyf(r, kExpm1));
  f2 s = add_f2f2(rr, q);
  s = add_f2_f(s, v);
  float p = pow2f(int_off(k));
  f2 t = add_f2_f(scale_f2(s, p), p);
  return norm_f2(add_f2_f(t, -1.0f));
}
__device__ __forceinline__ float copysignf_b(float v, uint32_t src) {
  return from_fbits((fbits(v) & ABS32) | (src & ~ABS32));
}
struct TanhU10 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x), ab = b & ABS32;
    float ac = ab < B91 ? from_fbits(ab) : 0.0f;
    f2 em = expm1_ff(__fmul_rn(2.0f, ac));
    f2 r = div_f2f2(em, add_f2_f(em, 2.0f));
    float y = __fadd_rn(r.x, r.y);
    if (!(ab < B91)) y = 1.0f;
    y = copysignf_b(y, b);
    if (ab > INF) y = from_fbits(QNAN32);
    return canonf(y);
  }
};
struct TanhU35 {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x), ab = b & ABS32;
    float ac = ab < B91 ? from_fbits(ab) : 0.0f;
    f2 em = expm1_ff(__fmul_rn(2.0f, ac));
    float e = __fadd_rn(em.x, em.y);
    float y = __fdiv_rn(e, __fadd_rn(e, 2.0f));
    if (!(ab < B91)) y = 1.0f;
    y = copysignf_b(y, b);
    if (ab > INF) y = from_fbits(QNAN32);
    return canonf(y);
  }
};

// e^(h + l) as FF for |h| <= 104 with a normal result
__device__ __forceinline__ f2 exp_ff(f2 a) {
  float k = rintf(__fmul_rn(a.x, R_LN2F));
  float h = __fmaf_rn(k, -L2AF, a.x);
  f2 r = add_ff(h, __fmaf_rn(k, -L2BF, a.y));
  float w = __fmaf_rn(__fmul_rn(r.x, r.x), polyf(r.x, kExpU10), r.y);
  f2 o = add_ff_fast(1.0f, r.x);
  return scale_f2(F2(o.x, __fadd_rn(o.y, w)), pow2f(int_off(k)));
}
__device__ __forceinline__ f2 erfc_tail(float ac) {   // erfc as FF for 1 <= ac < 3.95
  float u = __fsub_rn(ac, ERF_C);
  f2 e = add_f2f2(mul_ff(-ac, ac), F2(ERFB_C0H, ERFB_C0L));
  e = add_f2_f(e, __fmul_rn(u, polyf(u, kErfB)));
  return exp_ff(e);
}

struct ErfPaths {
  static constexpr int NCLS = 2;
  __device__ static int cls(float x) { return (fbits(x) & ABS32) >= B1; }
};
struct ErfU10 : ErfPaths {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x), ab = b & ABS32;
    float a = from_fbits(ab), y;
    if (ab < B1) {
      f2 t = mul_ff(a, a);
      float p = polyf(t.x, *reinterpret_cast<const float(*)[6]>(kErfA + 1));
      f2 w1 = add_ff_fast(kErfA[0], __fmul_rn(t.x, p));
      f2 w = add_f2f2_fast(F2(ERFA_C0H, ERFA_C0L), mul_f2f2(t, w1));
      f2 r = mul_f2_f(w, a);
      y = __fadd_rn(r.x, r.y);
      if (ab < 0x30800000u) {            // |x| < 2^-30: one rounding (subnormals)
        float as = __fmul_rn(a, 0x1p32f);
        y = __fmul_rn(__fmaf_rn(as, ERFA_C0H, __fmul_rn(as, ERFA_C0L)), 0x1p-32f);
      }
    } else {
      float ac = ab < B395 ? a : 1.0f;
      f2 c = erfc_tail(ac);
      f2 d = add_f_f2(1.0f, F2(-c.x, -c.y));
      y = __fadd_rn(d.x, d.y);
      if (!(ab < B395)) y = 1.0f;
    }
    y = copysignf_b(y, b);
    if (ab > INF) y = from_fbits(QNAN32);
    return canonf(y);
  }
};
struct ErfU35 : ErfPaths {
  __device__ float operator()(float x) const {
    uint32_t b = fbits(x), ab = b & ABS32;
    float a = from_fbits(ab), y;
    if (ab < B1) {
      float t = __fmul_rn(a, a);
      float p = __fmaf_rn(t, polyf(t, kErfA), ERFA_C0H);
      y = __fmul_rn(p, a);
    } else {
      float ac = ab < B395 ? a : 1.0f;
      f2 c = erfc_tail(ac);
      y = __fsub_rn(1.0f, __fadd_rn(c.x, c.y));
      if (!(ab < B395)) y = 1.0f;
    }
    y = copysignf_b(y, b);
    if (ab > INF) y = from_fbits(QNAN32);
    return canonf(y);
  }
};

}  // namespace explog32
}  // namespace sleefcu
