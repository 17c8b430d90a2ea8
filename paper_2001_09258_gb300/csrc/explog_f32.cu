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
// rounded to the 16-bit format with the hardware's round-to-nearest-even
// conversions (cvt.rn.bf16.f32 / cvt.rn.f16.f32, overflow to infinity,
// subnormal f16 results included); NaN results are the canonical 0x7FC0
// (bf16) / 0x7E00 (f16), chosen by a select.
//
// A 16-bit format has 65,536 inputs.  For large arrays each block first
// evaluates the functor on all of them into a 128 KB shared-memory table
// (the same FP32 body, so every entry is the bit pattern the direct form
// returns) and the array is then a gather through the table: the kernel is
// bounded by HBM traffic instead of by FP32 issue.  Small arrays evaluate
// directly (building a table costs as much as 65,536 elements per block).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <mutex>
namespace sleefcu {
namespace lowp {

__device__ __forceinline__ float bf16_in(uint16_t h) { return from_fbits((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t bf16_out(float f) {
  uint16_t r = __bfloat16_as_ushort(__float2bfloat16_rn(f));
  return (fbits(f) & ABS32) > EXP32 ? (uint16_t)0x7FC0 : r;
}
__device__ __forceinline__ float f16_in(uint16_t h) { return __half2float(__ushort_as_half(h)); }
__device__ __forceinline__ uint16_t f16_out(float f) {
  uint16_t r = __half_as_ushort(__float2half_rn(f));
  return (fbits(f) & ABS32) > EXP32 ? (uint16_t)0x7E00 : r;
}

template <class F, bool BF>
__device__ __forceinline__ uint16_t ev(const F &f, uint16_t h) {
  return BF ? bf16_out(f(bf16_in(h))) : f16_out(f(f16_in(h)));
}
// a packed pair (low half first), the conversions two at a time
template <class F, bool BF>
__device__ __forceinline__ uint32_t ev2(const F &f, uint32_t v) {
  float a, b;
  uint32_t r;
  if (BF) {
    a = f(bf16_in((uint16_t)(v & 0xFFFFu)));
    b = f(bf16_in((uint16_t)(v >> 16)));
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    r = *reinterpret_cast<uint32_t *>(&p);
    if ((fbits(a) & ABS32) > EXP32) r = (r & 0xFFFF0000u) | 0x7FC0u;
    if ((fbits(b) & ABS32) > EXP32) r = (r & 0x0000FFFFu) | 0x7FC00000u;
  } else {
    float2 in = __half22float2(*reinterpret_cast<const __half2 *>(&v));
    a = f(in.x);
    b = f(in.y);
    __half2 p = __floats2half2_rn(a, b);
    r = *reinterpret_cast<uint32_t *>(&p);
    if ((fbits(a) & ABS32) > EXP32) r = (r & 0xFFFF0000u) | 0x7E00u;
    if ((fbits(b) & ABS32) > EXP32) r = (r & 0x0000FFFFu) | 0x7E000000u;
  }
  return r;
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
      r.x = ev2<F, BF>(f, v.x);
      r.y = ev2<F, BF>(f, v.y);
      r.z = ev2<F, BF>(f, v.z);
      r.w = ev2<F, BF>(f, v.w);
      __stcs(o8 + i, r);
    }
    size_t rem = n & 7;
    if (tid < rem) out[n - rem + tid] = ev<F, BF>(f, x[n - rem + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = ev<F, BF>(f, x[i]);
  }
}

// the table form: one block per SM, 1024 threads
constexpr int kTabBlock = 1024;
constexpr size_t kTabMinN = (size_t)1 << 24;   // below this, direct evaluation
template <class F, bool BF>
__global__ void __launch_bounds__(kTabBlock, 1) k_lowp_table(const uint16_t *x, uint16_t *out, size_t n) {
  extern __shared__ uint32_t tab2[];           // 65,536 results as 32,768 packed pairs
  F f;
  for (uint32_t i = threadIdx.x; i < 32768u; i += kTabBlock) tab2[i] = ev2<F, BF>(f, (2u * i) | ((2u * i + 1u) << 16));
  __syncthreads();
  const uint16_t *tab = reinterpret_cast<const uint16_t *>(tab2);
  size_t stride = (size_t)gridDim.x * kTabBlock;
  size_t tid = (size_t)blockIdx.x * kTabBlock + threadIdx.x;
  size_t n8 = n >> 3;
  const uint4 *x8 = reinterpret_cast<const uint4 *>(x);
  uint4 *o8 = reinterpret_cast<uint4 *>(out);
  for (size_t i = tid; i < n8; i += stride) {
    uint4 v = __ldcs(x8 + i), r;
    r.x = tab[v.x & 0xFFFFu] | ((uint32_t)tab[v.x >> 16] << 16);
    r.y = tab[v.y & 0xFFFFu] | ((uint32_t)tab[v.y >> 16] << 16);
    r.z = tab[v.z & 0xFFFFu] | ((uint32_t)tab[v.z >> 16] << 16);
    r.w = tab[v.w & 0xFFFFu] | ((uint32_t)tab[v.w >> 16] << 16);
    __stcs(o8 + i, r);
  }
  size_t rem = n & 7;
  if (tid < rem) out[n - rem + tid] = tab[x[n - rem + tid]];
}

template <class F, bool BF>
sleefcu_status launch_lowp(const char *name, const void *x, void *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  const uint16_t *xi = (const uint16_t *)x;
  uint16_t *oi = (uint16_t *)out;
  if (sleefcu_status rc_ = check_args(name, n, xi, oi)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(out) && n >= kTabMinN) {
    auto k = k_lowp_table<F, BF>;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    static std::mutex mu;                      // 128 KB of dynamic shared memory is opt-in, per device
    static signed char attr[64];               // 0 not set yet, 1 set, -1 refused
    signed char a = -1;
    if (dev >= 0 && dev < 64) {
      std::lock_guard<std::mutex> lock(mu);
      if (attr[dev] == 0)
        attr[dev] = cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072) ==
                            cudaSuccess ? 1 : -1;
      a = attr[dev];
    }
    cudaGetLastError();
    if (a == 1) {
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      k<<<sms, kTabBlock, 131072, st>>>(xi, oi, n);
      return check_launch(name);
    }
  }
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
