// Device double-double (DD) and float-float (FF) operators.
//
// Table 5 of the paper ("DD Functions") names the operators; Section 5 keeps
// DD values un-normalized unless a step renormalizes them.  Every operator is
// a fixed sequence of IEEE round-to-nearest operations (the file is compiled
// with -fmad=false, so a product is fused into an add only where fma() is
// written), which is what makes the results identical to any other correct
// IEEE implementation of the same sequence (Section 4, bit-wise consistency).
#pragma once
#include <cuda_runtime.h>
#include "softfp64.cuh"

// Binary64 multiplication and rounding to an integral value (rint, trunc) in the kernels:
// exact software forms on the integer pipe (softfp64.cuh), bit-identical to
// the FP64 pipe's, so that the FP64 pipe, the bottleneck of the FP64 family
// on GB300, keeps only the additions and fused multiply-adds.  A translation
// unit chooses by defining SLEEFCU_SOFT_MUL before this header:
//   1 (default)  the software multiply inlined at each call site
//   2            one out-of-line copy of it, called from every site (large
//                kernels with many multiplications: the inlined copies cost
//                more instruction fetch than the call)
//   0            multiplications and roundings on the FP64 pipe
// All three give the same bits.
#ifndef SLEEFCU_SOFT_MUL
#define SLEEFCU_SOFT_MUL 1
#endif

namespace sleefcu {

#if SLEEFCU_SOFT_MUL == 2
static __device__ __noinline__ uint64_t dmul_call(uint64_t a, uint64_t b) { return soft::mul(a, b); }
#endif

__device__ __forceinline__ double dmul(double a, double b) {
#if SLEEFCU_SOFT_MUL == 2
  return __longlong_as_double((long long)dmul_call((uint64_t)__double_as_longlong(a),
                                                   (uint64_t)__double_as_longlong(b)));
#elif SLEEFCU_SOFT_MUL
  return __longlong_as_double((long long)soft::mul((uint64_t)__double_as_longlong(a),
                                                   (uint64_t)__double_as_longlong(b)));
#else
  return __dmul_rn(a, b);
#endif
}
__device__ __forceinline__ double drint(double a) {
#if SLEEFCU_SOFT_MUL
  return __longlong_as_double((long long)soft::rint((uint64_t)__double_as_longlong(a)));
#else
  return rint(a);
#endif
}
__device__ __forceinline__ double dtrunc(double a) {
#if SLEEFCU_SOFT_MUL
  return __longlong_as_double((long long)soft::trunc((uint64_t)__double_as_longlong(a)));
#else
  return trunc(a);
#endif
}

struct d2 { double x, y; };   // value x + y
struct f2 { float x, y; };

__device__ __forceinline__ d2 D2(double h, double l) { d2 r; r.x = h; r.y = l; return r; }
__device__ __forceinline__ f2 F2(float h, float l) { f2 r; r.x = h; r.y = l; return r; }

// ---- DD ----
// FastTwoSum, |a| >= |b|
__device__ __forceinline__ d2 add_dd_fast(double a, double b) {
  double s = __dadd_rn(a, b);
  return D2(s, __dadd_rn(__dsub_rn(a, s), b));
}
// TwoSum, any order
__device__ __forceinline__ d2 add_dd(double a, double b) {
  double s = __dadd_rn(a, b);
  double v = __dsub_rn(s, a);
  return D2(s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, v)), __dsub_rn(b, v)));
}
// DD + DD with |a| >= |b|
__device__ __forceinline__ d2 add_d2d2_fast(d2 a, d2 b) {
  double s = __dadd_rn(a.x, b.x);
  double t = __dadd_rn(__dsub_rn(a.x, s), b.x);
  return D2(s, __dadd_rn(__dadd_rn(t, a.y), b.y));
}
// DD + DD, any order
__device__ __forceinline__ d2 add_d2d2(d2 a, d2 b) {
  double s = __dadd_rn(a.x, b.x);
  double v = __dsub_rn(s, a.x);
  double e = __dadd_rn(__dsub_rn(a.x, __dsub_rn(s, v)), __dsub_rn(b.x, v));
  return D2(s, __dadd_rn(__dadd_rn(e, a.y), b.y));
}
// double + DD, |a| >= |b|
__device__ __forceinline__ d2 add_d_d2_fast(double a, d2 b) {
  double s = __dadd_rn(a, b.x);
  return D2(s, __dadd_rn(__dadd_rn(__dsub_rn(a, s), b.x), b.y));
}
// double + DD, any order
__device__ __forceinline__ d2 add_d_d2(double a, d2 b) {
  double s = __dadd_rn(a, b.x);
  double v = __dsub_rn(s, a);
  return D2(s, __dadd_rn(__dadd_rn(__dsub_rn(a, __dsub_rn(s, v)), __dsub_rn(b.x, v)), b.y));
}
// DD + double, |a| >= |b|
__device__ __forceinline__ d2 add_d2_d_fast(d2 a, double b) {
  double s = __dadd_rn(a.x, b);
  return D2(s, __dadd_rn(__dadd_rn(__dsub_rn(a.x, s), b), a.y));
}
// DD + double, any order
__device__ __forceinline__ d2 add_d2_d(d2 a, double b) {
  double s = __dadd_rn(a.x, b);
  double v = __dsub_rn(s, a.x);
  return D2(s, __dadd_rn(__dadd_rn(__dsub_rn(a.x, __dsub_rn(s, v)), __dsub_rn(b, v)), a.y));
}
// exact product: RN(ab) and the fma residual
__device__ __forceinline__ d2 mul_dd(double a, double b) {
  double s = dmul(a, b);
  return D2(s, __fma_rn(a, b, -s));
}
__device__ __forceinline__ d2 mul_d2_d(d2 a, double b) {
  double s = dmul(a.x, b);
  return D2(s, __fma_rn(a.y, b, __fma_rn(a.x, b, -s)));
}
__device__ __forceinline__ d2 mul_d2d2(d2 a, d2 b) {
  double s = dmul(a.x, b.x);
  return D2(s, __fma_rn(a.x, b.y, __fma_rn(a.y, b.x, __fma_rn(a.x, b.x, -s))));
}
__device__ __forceinline__ d2 sqr_d2(d2 a) {
  double s = dmul(a.x, a.x);
  return D2(s, __fma_rn(__dadd_rn(a.x, a.x), a.y, __fma_rn(a.x, a.x, -s)));
}
__device__ __forceinline__ d2 scale_d2(d2 a, double p2) { return D2(dmul(a.x, p2), dmul(a.y, p2)); }
__device__ __forceinline__ d2 norm_d2(d2 a) {
  double s = __dadd_rn(a.x, a.y);
  return D2(s, __dadd_rn(__dsub_rn(a.x, s), a.y));
}
// n / d with a single division
__device__ __forceinline__ d2 div_d2d2(d2 n, d2 d) {
  double t = __ddiv_rn(1.0, d.x);
  double q = dmul(n.x, t);
  double r = __fma_rn(-q, d.x, n.x);
  r = __fma_rn(-q, d.y, __dadd_rn(r, n.y));
  return D2(q, dmul(r, t));
}
__device__ __forceinline__ d2 rec_d(double d) {
  double t = __ddiv_rn(1.0, d);
  return D2(t, dmul(t, __fma_rn(-t, d, 1.0)));
}
__device__ __forceinline__ d2 rec_d2(d2 d) {
  double t = __ddiv_rn(1.0, d.x);
  double r = __fma_rn(-t, d.x, 1.0);
  r = __fma_rn(-t, d.y, r);
  return D2(t, dmul(r, t));
}
__device__ __forceinline__ d2 sqrt_d2(d2 a) {
  double h = __dsqrt_rn(a.x);
  double r = __dadd_rn(__fma_rn(-h, h, a.x), a.y);
  return D2(h, dmul(r, __ddiv_rn(1.0, __dadd_rn(h, h))));
}

// ---- FF (binary32) ----
__device__ __forceinline__ f2 add_ff_fast(float a, float b) {
  float s = __fadd_rn(a, b);
  return F2(s, __fadd_rn(__fsub_rn(a, s), b));
}
__device__ __forceinline__ f2 add_ff(float a, float b) {
  float s = __fadd_rn(a, b);
  float v = __fsub_rn(s, a);
  return F2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}
__device__ __forceinline__ f2 add_f2f2_fast(f2 a, f2 b) {
  float s = __fadd_rn(a.x, b.x);
  float t = __fadd_rn(__fsub_rn(a.x, s), b.x);
  return F2(s, __fadd_rn(__fadd_rn(t, a.y), b.y));
}
__device__ __forceinline__ f2 add_f2f2(f2 a, f2 b) {
  float s = __fadd_rn(a.x, b.x);
  float v = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
  return F2(s, __fadd_rn(__fadd_rn(e, a.y), b.y));
}
__device__ __forceinline__ f2 add_f_f2_fast(float a, f2 b) {
  float s = __fadd_rn(a, b.x);
  return F2(s, __fadd_rn(__fadd_rn(__fsub_rn(a, s), b.x), b.y));
}
__device__ __forceinline__ f2 add_f_f2(float a, f2 b) {
  float s = __fadd_rn(a, b.x);
  float v = __fsub_rn(s, a);
  return F2(s, __fadd_rn(__fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b.x, v)), b.y));
}
__device__ __forceinline__ f2 add_f2_f_fast(f2 a, float b) {
  float s = __fadd_rn(a.x, b);
  return F2(s, __fadd_rn(__fadd_rn(__fsub_rn(a.x, s), b), a.y));
}
__device__ __forceinline__ f2 add_f2_f(f2 a, float b) {
  float s = __fadd_rn(a.x, b);
  float v = __fsub_rn(s, a.x);
  return F2(s, __fadd_rn(__fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b, v)), a.y));
}
__device__ __forceinline__ f2 mul_ff(float a, float b) {
  float s = __fmul_rn(a, b);
  return F2(s, __fmaf_rn(a, b, -s));
}
__device__ __forceinline__ f2 mul_f2_f(f2 a, float b) {
  float s = __fmul_rn(a.x, b);
  return F2(s, __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -s)));
}
__device__ __forceinline__ f2 mul_f2f2(f2 a, f2 b) {
  float s = __fmul_rn(a.x, b.x);
  return F2(s, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -s))));
}
__device__ __forceinline__ f2 sqr_f2(f2 a) {
  float s = __fmul_rn(a.x, a.x);
  return F2(s, __fmaf_rn(__fadd_rn(a.x, a.x), a.y, __fmaf_rn(a.x, a.x, -s)));
}
__device__ __forceinline__ f2 scale_f2(f2 a, float p2) { return F2(__fmul_rn(a.x, p2), __fmul_rn(a.y, p2)); }
__device__ __forceinline__ f2 norm_f2(f2 a) {
  float s = __fadd_rn(a.x, a.y);
  return F2(s, __fadd_rn(__fsub_rn(a.x, s), a.y));
}
__device__ __forceinline__ f2 div_f2f2(f2 n, f2 d) {
  float t = __fdiv_rn(1.0f, d.x);
  float q = __fmul_rn(n.x, t);
  float r = __fmaf_rn(-q, d.x, n.x);
  r = __fmaf_rn(-q, d.y, __fadd_rn(r, n.y));
  return F2(q, __fmul_rn(r, t));
}
__device__ __forceinline__ f2 rec_f(float d) {
  float t = __fdiv_rn(1.0f, d);
  return F2(t, __fmul_rn(t, __fmaf_rn(-t, d, 1.0f)));
}
__device__ __forceinline__ f2 rec_f2(f2 d) {
  float t = __fdiv_rn(1.0f, d.x);
  float r = __fmaf_rn(-t, d.x, 1.0f);
  r = __fmaf_rn(-t, d.y, r);
  return F2(t, __fmul_rn(r, t));
}
__device__ __forceinline__ f2 sqrt_f2(f2 a) {
  float h = __fsqrt_rn(a.x);
  float r = __fadd_rn(__fmaf_rn(-h, h, a.x), a.y);
  return F2(h, __fdiv_rn(r, __fadd_rn(h, h)));
}

}  // namespace sleefcu
