// FP32 sin/cos cores (Cody-Waite, FF Payne-Hanek, polynomials) shared by the
// FP32 trigonometric entry points.
#pragma once
#include "sleefcu_common.cuh"
#include "sleefcu_phtab.inc"

namespace sleefcu {
namespace trig32 {

constexpr float PIO2F_A = 0x1.921fb6p0f, PIO2F_B = -0x1.777a5cp-25f;
constexpr float PIO2F_C = -0x1.ee59dap-50f, PIO2F_D = 0x1.98a2e0p-77f;
constexpr float R_1_PIF = 0x1.45f306p-2f;
constexpr float TWOPIF_H = 0x1.921fb6p2f, TWOPIF_L = -0x1.777a5cp-23f;
constexpr uint32_t B1 = 0x3f800000u, B125 = 0x42fa0000u, B2P20 = 0x49800000u;

constexpr float SIN_C1H = -0x1.5555560000000p-3f, SIN_C1L = 0x1.940bfe0000000p-28f;
static __constant__ float kSinU10[4] = {
  0x1.1111080000000p-7f, -0x1.a016880000000p-13f, 0x1.7147b00000000p-19f, -0x1.9704fc0000000p-26f};
static __constant__ float kSinU35[5] = {
  -0x1.5555560000000p-3f, 0x1.11112e0000000p-7f, -0x1.a01faa0000000p-13f, 0x1.7228ca0000000p-19f,
  -0x1.a61f4c0000000p-26f};

// float mod 4 of an integer-valued float, two's complement
__device__ __forceinline__ int q_of(float Q) { return low2_of_intf(Q); }

__device__ __forceinline__ f2 cw1(float x, float Q) {
  float u = __fmaf_rn(Q, -PIO2F_A, x);
  f2 s = add_f_f2(u, mul_ff(Q, -PIO2F_B));
  s.y = __fmaf_rn(Q, -PIO2F_C, s.y);
  return s;
}
__device__ __forceinline__ f2 cw1_exact(float x, float Q) {
  f2 s = add_f_f2(x, mul_ff(Q, -PIO2F_A));
  s = add_f2f2(s, mul_ff(Q, -PIO2F_B));
  s.y = __fmaf_rn(Q, -PIO2F_C, s.y);
  return s;
}
__device__ __forceinline__ f2 cw2(float x, float Q) {
  float u = __fmaf_rn(Q, -PIO2F_A, x);
  f2 s = add_f_f2(u, mul_ff(Q, -PIO2F_B));
  s = add_f2f2(s, mul_ff(Q, -PIO2F_C));
  s.y = __fmaf_rn(Q, -PIO2F_D, s.y);
  return s;
}

__device__ __forceinline__ void ph_step(f2 &x, int &q) {
  float r = rintf(__fmul_rn(4.0f, x.x));
  q += low2_of_intf(r);
  x.x = __fmaf_rn(r, -0.25f, x.x);
  x = norm_f2(x);
}
// Payne-Hanek in FF for |d| >= 2^20 or non-finite d
static __device__ __noinline__ f2 ph(float d, int &q) {
  uint32_t b = fbits(d);
  bool fin = (b & EXP32) != EXP32;
  uint32_t bf = fin ? b : 0u;
  int e = (int)((bf >> 23) & 0xFF) - 127;
  int sh = e > 64 ? 66 : 2;
  int ex = min(max(e, 0), 127);
  checked_note(fin && ex != e);         // a finite argument below 2^20 never comes here
  float u = bf ? from_fbits(bf - ((uint32_t)sh << 23)) : 0.0f;   // d * 2^-sh, exact
  float4 T = __ldg(reinterpret_cast<const float4 *>(k_phtab32 + 4 * ex));
  int qq = 0;
  f2 x = mul_ff(u, T.x);                 // (0,0) + y is y exactly
  ph_step(x, qq);
  x = add_f2f2(x, mul_ff(u, T.y));
  ph_step(x, qq);
  x = add_f2f2(x, mul_ff(u, T.z));
  ph_step(x, qq);
  x = add_f2f2(x, mul_ff(u, T.w));
  ph_step(x, qq);
  x = mul_f2f2(x, F2(TWOPIF_H, TWOPIF_L));
  uint32_t ib = (__ldg(k_phbit32 + (ex >> 5)) >> (ex & 31)) & 1u;
  q = (qq + 2 * (int)(bf & ib)) & 3;
  if (!fin) x.x = from_fbits(QNAN32);
  return x;
}
__device__ __forceinline__ f2 ph_fold(f2 r, int &q, int parity) {
  if ((q & 1) != parity) {
    bool ge = r.x >= 0.0f;
    float sa = ge ? -PIO2F_A : PIO2F_A, sb = ge ? -PIO2F_B : PIO2F_B;
    r = add_f2f2_fast(F2(sa, sb), r);
    q = (q + (ge ? 1 : -1)) & 3;
  }
  return r;
}

template <int PARITY>
__device__ __forceinline__ f2 reduce_half(float x, uint32_t ab, int &q) {
  if (ab < B2P20) {
    float k, Q;
    if (PARITY == 0) {
      k = rintf(__fmul_rn(x, R_1_PIF));
      Q = __fadd_rn(k, k);
    } else {
      k = rintf(__fmaf_rn(x, R_1_PIF, -0.5f));
      Q = __fmaf_rn(2.0f, k, 1.0f);
    }
    q = q_of(Q);
    if (PARITY == 1 && ab < B1) return cw1_exact(x, Q);
    if (ab < B125) return cw1(x, Q);
    return cw2(x, Q);
  }
  f2 r = ph(x, q);
  return ph_fold(r, q, PARITY);
}

__device__ __forceinline__ float sin_poly_u10(f2 s) {
  f2 t = sqr_f2(s);
  float p = polyf(t.x, kSinU10);
  f2 w = add_f2_f_fast(F2(SIN_C1H, SIN_C1L), __fmul_rn(t.x, p));
  w = mul_f2f2(t, w);
  w = mul_f2f2(s, w);
  f2 r = add_f2f2_fast(s, w);
  return __fadd_rn(r.x, r.y);
}
__device__ __forceinline__ float sin_poly_u35(float s) {
  float t = __fmul_rn(s, s);
  return __fmaf_rn(__fmul_rn(s, t), polyf(t, kSinU35), s);
}

// reduction path: 0 |x| < 125, 1 |x| < 2^20, 2 Payne-Hanek, 3 cos at |x| < 1
template <bool COS>
struct Paths {
  static constexpr int NCLS = COS ? 4 : 3;
  __device__ static int cls(float x) {
    uint32_t ab = fbits(x) & ABS32;
    if (COS && ab < B1) return 3;
    return ab < B125 ? 0 : (ab < B2P20 ? 1 : 2);
  }
  // the Payne-Hanek path (|x| >= 2^20 or non-finite) is deferred by the
  // plain binary32 kernel; 1.5 stands in for it on the Cody-Waite path
  static constexpr bool DEFER = true;
  static constexpr float kStandIn = 1.5f;
  __device__ static bool defer(float x) { return (fbits(x) & ABS32) >= B2P20; }
};

struct SinU10 : Paths<false> {
  __device__ float operator()(float x) const {
    uint32_t ab = fbits(x) & ABS32;
    int q;
    f2 s = reduce_half<0>(x, ab, q);
    float y = negf_if(sin_poly_u10(s), q & 2);
    if (ab == 0) y = x;
    return canonf(y);
  }
};
struct CosU10 : Paths<true> {
  __device__ float operator()(float x) const {
    uint32_t ab = fbits(x) & ABS32;
    int q;
    f2 s = reduce_half<1>(x, ab, q);
    return canonf(negf_if(sin_poly_u10(s), !(q & 2)));
  }
};
struct SinU35 : Paths<false> {
  __device__ float operator()(float x) const {
    uint32_t ab = fbits(x) & ABS32;
    int q;
    f2 s = reduce_half<0>(x, ab, q);
    float y = negf_if(sin_poly_u35(__fadd_rn(s.x, s.y)), q & 2);
    if (ab == 0) y = x;
    return canonf(y);
  }
};
struct CosU35 : Paths<true> {
  __device__ float operator()(float x) const {
    uint32_t ab = fbits(x) & ABS32;
    int q;
    f2 s = reduce_half<1>(x, ab, q);
    return canonf(negf_if(sin_poly_u35(__fadd_rn(s.x, s.y)), !(q & 2)));
  }
};

}  // namespace trig32
}  // namespace sleefcu
