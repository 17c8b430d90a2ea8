// FP32 exp, log, log1p, tanh, erf (u10, u35) for sm_103a, binary32 only.
//
// exp: Section 5.6 in binary32, u10 keeping the residual of the reduced
//   argument and forming 1 + r in float-float (FF).
// log / log1p: Section 5.5 in binary32; log1p first forms 1 + x as an FF
//   pair and applies the reduction to the pair.
// tanh: expm1(2|x|) / (expm1(2|x|) + 2) in FF.
// erf: |x| < 1: x (c0 + t (c1 + t P(t))) with the two leading terms in FF;
//   1 <= |x| < 3.95: 1 - exp(-x^2 + L), L = log(erfc(x) e^(x^2)) a polynomial
//   in |x| - 2.475, the exponent and the exponential in FF.
// Plain 16-byte vectorized kernels (for binary32 the divergence-sorted tiles
// cost about what they save).
#include "explog32_core.cuh"

// ---------------- bf16 / f16 forms ----------------
// 16-bit input converted exactly to binary32, the FP32 functor, the result
// rounded to the 16-bit format (round-to-nearest-even, integer arithmetic);
// NaN results are the canonical 0x7FC0 (bf16) / 0x7E00 (f16).
namespace sleefcu {
namespace lowp {

__device__ __forceinline__ float bf16_in(uint16_t h) { return from_fbits((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t bf16_out(float f) {
  uint32_t b = fbits(f);
  if ((b & ABS32) > EXP32) return 0x7FC0;
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
__device__ __forceinline__ float f16_in(uint16_t h) {
  uint32_t s = (uint32_t)(h & 0x8000u) << 16, e = (h >> 10) & 0x1Fu, m = h & 0x3FFu;
  if (e == 0x1F) return from_fbits(s | 0x7F800000u | (m << 13));
  if (e) return from_fbits(s | ((e + 112u) << 23) | (m << 13));
  float f = __fmul_rn(__uint2float_rn(m), 0x1p-24f);     // exact
  return s ? -f : f;
}
__device__ __forceinline__ uint16_t f16_out(float f) {
  uint32_t b = fbits(f), sign = (b >> 16) & 0x8000u, ab = b & ABS32;
  if (ab > EXP32) return 0x7E00;
  if (ab >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u);
  if (ab >= 0x38800000u) {
    uint32_t r = ab - (112u << 23);
    r += 0xFFFu + ((r >> 13) & 1u);
    return (uint16_t)(sign | (r >> 13));
  }
  uint32_t t = fbits(__fadd_rn(from_fbits(ab), 0.5f)) - 0x3F000000u;   // RNE to 2^-24 units
  return (uint16_t)(sign | t);
}

template <class F, bool BF>
__device__ __forceinline__ uint16_t ev(const F &f, uint16_t h) {
  return BF ? bf16_out(f(bf16_in(h))) : f16_out(f(f16_in(h)));
}

template <class F, bool BF, bool VEC>
__global__ void __launch_bounds__(kBlock) k_lowp(const uint16_t *x, uint16_t *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t n8 = n >> 3;
    const uint4 *x8 = reinterpret_cast<const uint4 *>(x);
    uint4 *o8 = reinterpret_cast<uint4 *>(out);
    for (size_t i = tid; i < n8; i += stride) {
      uint4 v = __ldcs(x8 + i), r;
      r.x = ev<F, BF>(f, (uint16_t)(v.x & 0xFFFF)) | ((uint32_t)ev<F, BF>(f, (uint16_t)(v.x >> 16)) << 16);
      r.y = ev<F, BF>(f, (uint16_t)(v.y & 0xFFFF)) | ((uint32_t)ev<F, BF>(f, (uint16_t)(v.y >> 16)) << 16);
      r.z = ev<F, BF>(f, (uint16_t)(v.z & 0xFFFF)) | ((uint32_t)ev<F, BF>(f, (uint16_t)(v.z >> 16)) << 16);
      r.w = ev<F, BF>(f, (uint16_t)(v.w & 0xFFFF)) | ((uint32_t)ev<F, BF>(f, (uint16_t)(v.w >> 16)) << 16);
      __stcs(o8 + i, r);
    }
    size_t rem = n & 7;
    if (tid < rem) out[n - rem + tid] = ev<F, BF>(f, x[n - rem + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = ev<F, BF>(f, x[i]);
  }
}

template <class F, bool BF>
sleefcu_status launch_lowp(const char *name, const void *x, void *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  const uint16_t *xi = (const uint16_t *)x;
  uint16_t *oi = (uint16_t *)out;
  if (sleefcu_status rc_ = check_args(name, n, xi, oi)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(out)) {
    auto k = k_lowp<F, BF, true>;
    k<<<grid_for((const void *)k, (n + 7) / 8), kBlock, 0, st>>>(xi, oi, n);
  } else {
    auto k = k_lowp<F, BF, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(xi, oi, n);
  }
  return check_launch(name);
}

}  // namespace lowp
}  // namespace sleefcu


#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

#define UNARY32(NAME, F)                                                                    \
  extern "C" sleefcu_status sleefcu_##NAME(const float *x, float *out, size_t n,            \
                                           sleefcu_stream s) {                              \
    return launch_unary32<explog32::F>("sleefcu_" #NAME, x, out, n, s);                     \
  }
UNARY32(exp_u10_f32, ExpU10)
UNARY32(exp_u35_f32, ExpU35)
UNARY32(log_u10_f32, LogU10)
UNARY32(log_u35_f32, LogU35)
UNARY32(log1p_u10_f32, Log1pU10)
UNARY32(log1p_u35_f32, Log1pU35)
UNARY32(tanh_u10_f32, TanhU10)
UNARY32(tanh_u35_f32, TanhU35)
extern "C" sleefcu_status sleefcu_erf_u10_f32(const float *x, float *out, size_t n, sleefcu_stream s) {
  return launch_unary32<explog32::ErfU10>("sleefcu_erf_u10_f32", x, out, n, s);
}
extern "C" sleefcu_status sleefcu_erf_u35_f32(const float *x, float *out, size_t n, sleefcu_stream s) {
  return launch_unary32<explog32::ErfU35>("sleefcu_erf_u35_f32", x, out, n, s);
}

#define LOWP(NAME, F)                                                                       \
  extern "C" sleefcu_status sleefcu_##NAME##_bf16(const void *x, void *out, size_t n,       \
                                                  sleefcu_stream s) {                       \
    return lowp::launch_lowp<explog32::F, true>("sleefcu_" #NAME "_bf16", x, out, n, s);    \
  }                                                                                         \
  extern "C" sleefcu_status sleefcu_##NAME##_f16(const void *x, void *out, size_t n,        \
                                                 sleefcu_stream s) {                        \
    return lowp::launch_lowp<explog32::F, false>("sleefcu_" #NAME "_f16", x, out, n, s);    \
  }
LOWP(erf_u10, ErfU10)
LOWP(erf_u35, ErfU35)
LOWP(tanh_u10, TanhU10)
LOWP(tanh_u35, TanhU35)
LOWP(exp_u10, ExpU10)
LOWP(exp_u35, ExpU35)
LOWP(log1p_u10, Log1pU10)
LOWP(log1p_u35, Log1pU35)
#undef UNARY32
#undef LOWP
#endif  // SLEEFCU_FUNCTORS_ONLY
