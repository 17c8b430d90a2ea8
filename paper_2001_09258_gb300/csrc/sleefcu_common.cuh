// Shared device helpers and the elementwise launch machinery of libsleefcu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>
#include <stddef.h>
#include "../../include/sleefcu.h"
#include "sleefcu_dd.cuh"

namespace sleefcu {

// ---------------- checked build: device error word ----------------
// In the checked build each translation unit keeps a counter of table
// indices that had to be clamped for a finite argument (a lane that reached
// a table gather it should never reach); the kernels count and go on, they
// never trap.  sleefcu_checked_error_count() sums the counters of all units.
#ifdef SLEEFCU_CHECKED
static __device__ unsigned long long g_checked_count;
void register_checked_word(sleefcu_status (*read)(unsigned long long *, int));
namespace {
sleefcu_status read_checked_word(unsigned long long *v, int reset) {
  unsigned long long x = 0;
  if (cudaMemcpyFromSymbol(&x, g_checked_count, sizeof x) != cudaSuccess) return SLEEFCU_ECUDA;
  if (reset) {
    const unsigned long long z = 0;
    if (cudaMemcpyToSymbol(g_checked_count, &z, sizeof z) != cudaSuccess) return SLEEFCU_ECUDA;
  }
  *v += x;
  return SLEEFCU_OK;
}
struct CheckedWordReg {
  CheckedWordReg() { register_checked_word(&read_checked_word); }
} g_checked_word_reg;
}  // namespace
__device__ __forceinline__ void checked_note(bool bad) {
  if (bad) atomicAdd(&g_checked_count, 1ull);
}
#else
__device__ __forceinline__ void checked_note(bool) {}
#endif

// ---------------- bit helpers (integer pipe) ----------------
// The bits of a double through an opaque register move: the compiler would
// otherwise turn NaN, infinity and sign tests written on the bits back into
// FP64 comparisons, and on GB300 each takes an FP64-pipe slot like an FMA.
__device__ __forceinline__ uint64_t bits(double d) {
  uint64_t r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(d));
  return r;
}
__device__ __forceinline__ double from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint32_t fbits(float f) { return (uint32_t)__float_as_uint(f); }
__device__ __forceinline__ float from_fbits(uint32_t b) { return __uint_as_float(b); }
__device__ __forceinline__ double neg_if(double v, bool c) { return from_bits(bits(v) ^ ((uint64_t)c << 63)); }
__device__ __forceinline__ float negf_if(float v, bool c) { return from_fbits(fbits(v) ^ ((uint32_t)c << 31)); }
constexpr uint64_t ABS64 = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t EXP64 = 0x7FF0000000000000ull;
constexpr uint64_t QNAN64 = 0x7FF8000000000000ull;
constexpr uint32_t ABS32 = 0x7FFFFFFFu;
constexpr uint32_t EXP32 = 0x7F800000u;
constexpr uint32_t QNAN32 = 0x7FC00000u;
__device__ __forceinline__ bool is_nan_b(uint64_t b) { return (b & ABS64) > EXP64; }
__device__ __forceinline__ bool is_finite_b(uint64_t b) { return (b & EXP64) != EXP64; }
// canonical quiet NaN for any NaN result
__device__ __forceinline__ double canon(double y) { return is_nan_b(bits(y)) ? from_bits(QNAN64) : y; }
__device__ __forceinline__ float canonf(float y) {
  return (fbits(y) & ABS32) > EXP32 ? from_fbits(QNAN32) : y;
}

// Comparisons of a double with a constant on the integer pipe: on GB300 an
// FP64 comparison occupies an FP64-pipe slot like an FMA.  okey() increases
// with the value over all non-NaN doubles (-0 sorts just below +0); with a
// non-zero constant c each helper returns the IEEE result for every x, NaNs
// included.
__device__ __forceinline__ long long okey(double d) {
  long long b = (long long)bits(d);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ bool not_nan(double d) { return (bits(d) & ABS64) <= EXP64; }
__device__ __forceinline__ bool lt_c(double x, double c) { return not_nan(x) && okey(x) < okey(c); }
__device__ __forceinline__ bool le_c(double x, double c) { return not_nan(x) && okey(x) <= okey(c); }
__device__ __forceinline__ bool gt_c(double x, double c) { return not_nan(x) && okey(x) > okey(c); }
__device__ __forceinline__ bool ge_c(double x, double c) { return not_nan(x) && okey(x) >= okey(c); }
// x < 0, x > 0 and x == 0 with IEEE semantics (signed zeros equal, NaN false)
__device__ __forceinline__ bool lt_0(double x) { return (bits(x) >> 63) && (bits(x) & ABS64) - 1 < EXP64; }
__device__ __forceinline__ bool gt_0(double x) { return !(bits(x) >> 63) && bits(x) - 1 < EXP64; }
__device__ __forceinline__ bool eq_0(double x) { return (bits(x) & ABS64) == 0; }

// a finite |x|, given as its bits, is an integer / an odd integer
__device__ __forceinline__ bool integral_b(uint64_t ab) {
  int e = (int)(ab >> 52) - 1023;
  if (e >= 52) return true;
  if (e < 0) return ab == 0;
  return (ab & ((1ull << (52 - e)) - 1)) == 0;
}
__device__ __forceinline__ bool odd_int_b(uint64_t ab) {
  int e = (int)(ab >> 52) - 1023;
  if (e < 0 || e > 52) return false;
  uint64_t m = (ab & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  return integral_b(ab) && ((m >> (52 - e)) & 1);
}

// For an integer-valued double k (|k| < 2^63 or a multiple of 4 above),
// k mod 4 in two's complement, computed on the integer pipe.
__device__ __forceinline__ int low2_of_int(double k) {
  uint64_t b = bits(k);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  uint64_t iv = e < 0 ? 0 : (e <= 52 ? (m >> (52 - e)) : (e < 64 ? (m << (e - 52)) : 0));
  int v = (int)(iv & 3);
  return (b >> 63) ? ((-v) & 3) : v;
}
__device__ __forceinline__ int low2_of_intf(float k) {
  uint32_t b = fbits(k);
  int e = (int)((b >> 23) & 0xFF) - 127;
  uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
  uint32_t iv = e < 0 ? 0 : (e <= 23 ? (m >> (23 - e)) : (e < 32 ? (m << (e - 23)) : 0));
  int v = (int)(iv & 3);
  return (b >> 31) ? ((-v) & 3) : v;
}

// ---------------- Estrin's scheme ----------------
// E(c, n) = c[0] for n = 1, else fma(t^m, E(c+m, n-m), E(c, m)) with m the
// largest power of two below n (Section 5's polynomial evaluation).  pw[k]
// holds t^(2^k).
template <int N>
struct Estrin {
  static constexpr int M = (N <= 2) ? 1 : (N <= 4) ? 2 : (N <= 8) ? 4 : (N <= 16) ? 8 : 16;
  static constexpr int K = (M == 1) ? 0 : (M == 2) ? 1 : (M == 4) ? 2 : (M == 8) ? 3 : 4;
  __device__ __forceinline__ static double d(const double *c, const double *pw) {
    return __fma_rn(pw[K], Estrin<N - M>::d(c + M, pw), Estrin<M>::d(c, pw));
  }
  __device__ __forceinline__ static float f(const float *c, const float *pw) {
    return __fmaf_rn(pw[K], Estrin<N - M>::f(c + M, pw), Estrin<M>::f(c, pw));
  }
};
template <>
struct Estrin<1> {
  __device__ __forceinline__ static double d(const double *c, const double *) { return c[0]; }
  __device__ __forceinline__ static float f(const float *c, const float *) { return c[0]; }
};
template <int N>
__device__ __forceinline__ double poly(double t, const double (&c)[N]) {
  double pw[5];
  pw[0] = t;
  if (N > 2) pw[1] = dmul(t, t);
  if (N > 4) pw[2] = dmul(pw[1], pw[1]);
  if (N > 8) pw[3] = dmul(pw[2], pw[2]);
  if (N > 16) pw[4] = dmul(pw[3], pw[3]);
  return Estrin<N>::d(c, pw);
}
// the same for N coefficients starting at c (a row of a table)
template <int N>
__device__ __forceinline__ double poly_p(double t, const double *c) {
  double pw[5];
  pw[0] = t;
  if (N > 2) pw[1] = dmul(t, t);
  if (N > 4) pw[2] = dmul(pw[1], pw[1]);
  if (N > 8) pw[3] = dmul(pw[2], pw[2]);
  if (N > 16) pw[4] = dmul(pw[3], pw[3]);
  return Estrin<N>::d(c, pw);
}
template <int N>
__device__ __forceinline__ float polyf(float t, const float (&c)[N]) {
  float pw[5];
  pw[0] = t;
  if (N > 2) pw[1] = __fmul_rn(t, t);
  if (N > 4) pw[2] = __fmul_rn(pw[1], pw[1]);
  if (N > 8) pw[3] = __fmul_rn(pw[2], pw[2]);
  if (N > 16) pw[4] = __fmul_rn(pw[3], pw[3]);
  return Estrin<N>::f(c, pw);
}

// ---------------- elementwise kernels ----------------
constexpr int kBlock = 256;

// unary: out[i] = F(x[i]); VEC processes pairs with 16-byte accesses
template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_unary64(const double *x, double *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t np = n >> 1;
    const double2 *x2 = reinterpret_cast<const double2 *>(x);
    double2 *o2 = reinterpret_cast<double2 *>(out);
    for (size_t i = tid; i < np; i += stride) {
      double2 v = __ldcs(x2 + i);
      double2 r;
      r.x = f(v.x);
      r.y = f(v.y);
      __stcs(o2 + i, r);
    }
    if ((n & 1) && tid == 0) out[n - 1] = f(x[n - 1]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i]);
  }
}

template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_binary64(const double *x, const double *y, double *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t np = n >> 1;
    const double2 *x2 = reinterpret_cast<const double2 *>(x);
    const double2 *y2 = reinterpret_cast<const double2 *>(y);
    double2 *o2 = reinterpret_cast<double2 *>(out);
    for (size_t i = tid; i < np; i += stride) {
      double2 a = __ldcs(x2 + i), b = __ldcs(y2 + i);
      double2 r;
      r.x = f(a.x, b.x);
      r.y = f(a.y, b.y);
      __stcs(o2 + i, r);
    }
    if ((n & 1) && tid == 0) out[n - 1] = f(x[n - 1], y[n - 1]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i], y[i]);
  }
}

// two outputs (sincos): F::operator()(x, &a, &b)
template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_dual64(const double *x, double *o1, double *o2, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t np = n >> 1;
    const double2 *x2 = reinterpret_cast<const double2 *>(x);
    double2 *a2 = reinterpret_cast<double2 *>(o1);
    double2 *b2 = reinterpret_cast<double2 *>(o2);
    for (size_t i = tid; i < np; i += stride) {
      double2 v = __ldcs(x2 + i);
      double2 a, b;
      f(v.x, a.x, b.x);
      f(v.y, a.y, b.y);
      __stcs(a2 + i, a);
      __stcs(b2 + i, b);
    }
    if ((n & 1) && tid == 0) f(x[n - 1], o1[n - 1], o2[n - 1]);
  } else {
    for (size_t i = tid; i < n; i += stride) f(x[i], o1[i], o2[i]);
  }
}

// ---------------- divergence-sorted tiles ----------------
// For functions whose lanes take different paths (Cody-Waite level 1 or 2,
// Payne-Hanek, ...), a CTA loads a tile, classifies every element with
// F::cls, scatters the elements into shared memory grouped by class and
// evaluates them in that order, so that each warp runs one path; results are
// gathered back and stored coalesced.  The arithmetic per element is
// unchanged, so the output bits do not depend on the grouping.
constexpr int kSortEPT = 4;
constexpr int kSortTile = kBlock * kSortEPT;

// elements per thread of a functor's sorted tiles: F::SORT_EPT where the
// functor sets it (many classes, some small: a larger tile leaves fewer warps
// straddling two classes), else kSortEPT
template <class F, class = void>
struct sort_ept { static constexpr int value = kSortEPT; };
template <class F>
struct sort_ept<F, std::void_t<decltype(F::SORT_EPT)>> { static constexpr int value = F::SORT_EPT; };
// resident blocks per SM the sorted kernel of F is compiled for (its
// register budget): F::MIN_BLOCKS if given, else 1
template <class F, class = void>
struct sort_minb { static constexpr int value = 1; };
template <class F>
struct sort_minb<F, std::void_t<decltype(F::MIN_BLOCKS)>> { static constexpr int value = F::MIN_BLOCKS; };

template <int NC, int EPT>
__device__ __forceinline__ void sort_scatter(const int (&cl)[EPT], int *cur, unsigned short *sidx, int tid) {
  const unsigned lane = tid & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int j = 0; j < EPT; j++) {
    if constexpr (NC > 4) {
      // many classes: the lanes of one class find each other with a match
      // instead of one ballot per class
      unsigned m = __match_any_sync(0xffffffffu, cl[j]);
      int leader = __ffs(m) - 1;
      int b = 0;
      if ((int)lane == leader && cl[j] >= 0) b = atomicAdd(&cur[cl[j]], __popc(m));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (cl[j] >= 0) sidx[b + __popc(m & lt)] = (unsigned short)(j * kBlock + tid);
    } else {
#pragma unroll
      for (int c = 0; c < NC; c++) {
        unsigned m = __ballot_sync(0xffffffffu, cl[j] == c);
        if (m) {
          int b = 0;
          if (lane == 0) b = atomicAdd(&cur[c], __popc(m));
          b = __shfl_sync(0xffffffffu, b, 0);
          if (cl[j] == c) sidx[b + __popc(m & lt)] = (unsigned short)(j * kBlock + tid);
        }
      }
    }
  }
}

template <int NC, int EPT>
__device__ __forceinline__ void sort_count(const int (&cl)[EPT], int *cnt, int tid) {
  const unsigned lane = tid & 31;
  for (int j = 0; j < EPT; j++) {
    if constexpr (NC > 4) {
      unsigned m = __match_any_sync(0xffffffffu, cl[j]);
      if ((int)lane == __ffs(m) - 1 && cl[j] >= 0) atomicAdd(&cnt[cl[j]], __popc(m));
    } else {
#pragma unroll
      for (int c = 0; c < NC; c++) {
        unsigned m = __ballot_sync(0xffffffffu, cl[j] == c);
        if (lane == 0 && m) atomicAdd(&cnt[c], __popc(m));
      }
    }
  }
}

// unary (NOUT = 1) or one-input-two-output (NOUT = 2) sorted kernel; each
// result overwrites its staged argument (a sorted position belongs to one
// thread), the second output of NOUT = 2 has its own buffer
//
// MASKED: only the elements whose mask byte is non-zero are classified,
// evaluated (densely, as the tile's sorted prefix) and stored; the other
// outputs are left untouched (the masked entry points).
template <class F, int NOUT, bool MASKED = false>
__global__ void __launch_bounds__(kBlock, sort_minb<F>::value) k_sorted64(const double *x, double *o1, double *o2, size_t n,
                                                     const uint8_t *mask = nullptr) {
  constexpr int NC = F::NCLS, EPT = sort_ept<F>::value, TILE = kBlock * EPT;
  __shared__ double sx[TILE];
  __shared__ double so2[NOUT == 2 ? TILE : 1];
  __shared__ unsigned short sidx[TILE];
  __shared__ int cnt[NC], cur[NC], tot;
  F f;
  const int tid = threadIdx.x;
  const size_t ntiles = (n + TILE - 1) / TILE;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * TILE;
    const int valid = (int)((n - base) < (size_t)TILE ? (n - base) : (size_t)TILE);
    if (tid < NC) cnt[tid] = 0;
    __syncthreads();
    int cl[EPT];
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      double v = 0.0;
      cl[j] = -1;
      if (e < valid && (!MASKED || mask[base + e])) {
        v = __ldcs(x + base + e);
        cl[j] = F::cls(v);
      }
      sx[e] = v;
    }
    sort_count<NC, EPT>(cl, cnt, tid);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int c = 0; c < NC; c++) { cur[c] = acc; acc += cnt[c]; }
      tot = acc;
    }
    __syncthreads();
    sort_scatter<NC, EPT>(cl, cur, sidx, tid);
    __syncthreads();
    const int m = MASKED ? tot : valid;
    for (int k = tid; k < m; k += kBlock) {
      int e = sidx[k];
      if constexpr (NOUT == 1) {
        sx[e] = f(sx[e]);
      } else {
        double a, b;
        f.dual(sx[e], a, b);
        sx[e] = a;
        so2[e] = b;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      if (e < valid && (!MASKED || mask[base + e])) {
        __stcs(o1 + base + e, sx[e]);
        if constexpr (NOUT == 2) __stcs(o2 + base + e, so2[e]);
      }
    }
    __syncthreads();
  }
}

// binary sorted kernel: class from (x, y)
template <class F, bool MASKED = false>
__global__ void __launch_bounds__(kBlock) k_sorted64b(const double *x, const double *y, double *o, size_t n,
                                                      const uint8_t *mask = nullptr) {
  constexpr int NC = F::NCLS, EPT = sort_ept<F>::value, TILE = kBlock * EPT;
  __shared__ double sx[TILE];
  __shared__ double sy[TILE];
  __shared__ unsigned short sidx[TILE];
  __shared__ int cnt[NC], cur[NC], tot;
  F f;
  const int tid = threadIdx.x;
  const size_t ntiles = (n + TILE - 1) / TILE;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * TILE;
    const int valid = (int)((n - base) < (size_t)TILE ? (n - base) : (size_t)TILE);
    if (tid < NC) cnt[tid] = 0;
    __syncthreads();
    int cl[EPT];
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      double a = 0.0, b = 0.0;
      if (e < valid && (!MASKED || mask[base + e])) {
        a = __ldcs(x + base + e);
        b = __ldcs(y + base + e);
        cl[j] = F::cls(a, b);
      } else {
        cl[j] = -1;
      }
      sx[e] = a;
      sy[e] = b;
    }
    sort_count<NC, EPT>(cl, cnt, tid);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int c = 0; c < NC; c++) { cur[c] = acc; acc += cnt[c]; }
      tot = acc;
    }
    __syncthreads();
    sort_scatter<NC, EPT>(cl, cur, sidx, tid);
    __syncthreads();
    const int m = MASKED ? tot : valid;
    for (int k = tid; k < m; k += kBlock) {
      int e = sidx[k];
      double r = f(sx[e], sy[e]);
      sx[e] = r;   // each e is owned by exactly one k
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      if (e < valid && (!MASKED || mask[base + e])) __stcs(o + base + e, sx[e]);
    }
    __syncthreads();
  }
}

// ---------------- host side ----------------
void set_error(const char *fmt, ...);
sleefcu_status check_launch(const char *what);
int grid_for(const void *kernel, size_t work_items);

// Argument checks of the checked build (-DSLEEFCU_CHECKED, libsleefcu_checked.so):
// every device array of a call must be device (or managed) memory of the
// current device holding its n elements; otherwise the call returns
// SLEEFCU_EINVAL before any launch.  In the normal build the check is empty.
#ifdef SLEEFCU_CHECKED
sleefcu_status check_dev_range(const char *name, const void *p, size_t bytes);
template <class... P>
sleefcu_status check_args(const char *name, size_t n, const P *...p) {
  sleefcu_status r = SLEEFCU_OK;
  ((r = (r == SLEEFCU_OK ? check_dev_range(name, (const void *)p, n * sizeof(P)) : r)), ...);
  return r;
}
#else
template <class... P>
constexpr sleefcu_status check_args(const char *, size_t, const P *...) { return SLEEFCU_OK; }
#endif

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

template <class F>
sleefcu_status launch_unary64(const char *name, const double *x, double *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(out)) {
    auto k = k_unary64<F, true>;
    k<<<grid_for((const void *)k, (n + 1) / 2), kBlock, 0, st>>>(x, out, n);
  } else {
    auto k = k_unary64<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, out, n);
  }
  return check_launch(name);
}

template <class F>
sleefcu_status launch_binary64(const char *name, const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !y || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, y, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(y) && aligned16(out)) {
    auto k = k_binary64<F, true>;
    k<<<grid_for((const void *)k, (n + 1) / 2), kBlock, 0, st>>>(x, y, out, n);
  } else {
    auto k = k_binary64<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, y, out, n);
  }
  return check_launch(name);
}

template <class F>
sleefcu_status launch_dual64(const char *name, const double *x, double *o1, double *o2, size_t n,
                             sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !o1 || !o2) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, o1, o2)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(o1) && aligned16(o2)) {
    auto k = k_dual64<F, true>;
    k<<<grid_for((const void *)k, (n + 1) / 2), kBlock, 0, st>>>(x, o1, o2, n);
  } else {
    auto k = k_dual64<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, o1, o2, n);
  }
  return check_launch(name);
}

template <class F>
sleefcu_status launch_sorted64(const char *name, const double *x, double *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, out)) return rc_;
  auto k = k_sorted64<F, 1>;
  constexpr int EPT = sort_ept<F>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, out, out, n, nullptr);
  return check_launch(name);
}
template <class F>
sleefcu_status launch_sorted64_dual(const char *name, const double *x, double *o1, double *o2, size_t n,
                                    sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !o1 || !o2) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, o1, o2)) return rc_;
  auto k = k_sorted64<F, 2>;
  constexpr int EPT = sort_ept<F>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, o1, o2, n, nullptr);
  return check_launch(name);
}
template <class F>
sleefcu_status launch_sorted64b(const char *name, const double *x, const double *y, double *out, size_t n,
                                sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !y || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, y, out)) return rc_;
  auto k = k_sorted64b<F>;
  constexpr int EPT = sort_ept<F>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, y, out, n, nullptr);
  return check_launch(name);
}

// ---- masked entry points (the paper's whole-function opmask) ----
// A functor without path classes is sorted as one class, so that the
// selected elements are still evaluated densely.
template <class F, class = void>
struct has_classes : std::false_type {};
template <class F>
struct has_classes<F, std::void_t<decltype(F::NCLS)>> : std::true_type {};
template <class F>
struct OneClass : F {
  static constexpr int NCLS = 1;
  __device__ static int cls(double) { return 0; }
  __device__ static int cls(double, double) { return 0; }
};
template <class F>
using sortable_t = typename std::conditional<has_classes<F>::value, F, OneClass<F>>::type;

template <class F>
sleefcu_status launch_masked64(const char *name, const double *x, const uint8_t *mask, double *out, size_t n,
                               sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !mask || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, mask, out)) return rc_;
  using G = sortable_t<F>;
  auto k = k_sorted64<G, 1, true>;
  constexpr int EPT = sort_ept<G>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, out, out, n, mask);
  return check_launch(name);
}
template <class F>
sleefcu_status launch_masked64_dual(const char *name, const double *x, const uint8_t *mask, double *o1,
                                    double *o2, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !mask || !o1 || !o2) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, mask, o1, o2)) return rc_;
  using G = sortable_t<F>;
  auto k = k_sorted64<G, 2, true>;
  constexpr int EPT = sort_ept<G>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, o1, o2, n, mask);
  return check_launch(name);
}
template <class F>
sleefcu_status launch_masked64b(const char *name, const double *x, const double *y, const uint8_t *mask,
                                double *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !y || !mask || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, y, mask, out)) return rc_;
  using G = sortable_t<F>;
  auto k = k_sorted64b<G, true>;
  constexpr int EPT = sort_ept<G>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, y, out, n, mask);
  return check_launch(name);
}

}  // namespace sleefcu

// ---------------- FP32 kernels ----------------
namespace sleefcu {

// unary FP32: out[i] = F(x[i]); VEC processes 4 elements per 16-byte access
template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_unary32(const float *x, float *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t nq = n >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    for (size_t i = tid; i < nq; i += stride) {
      float4 v = __ldcs(x4 + i);
      float4 r;
      r.x = f(v.x);
      r.y = f(v.y);
      r.z = f(v.z);
      r.w = f(v.w);
      __stcs(o4 + i, r);
    }
    size_t rem = n & 3;
    if (tid < rem) out[n - rem + tid] = f(x[n - rem + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i]);
  }
}

// FP32 divergence-sorted tiles (see k_sorted64)
template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_binary32(const float *x, const float *y, float *out, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t nq = n >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    for (size_t i = tid; i < nq; i += stride) {
      float4 a = __ldcs(x4 + i), b = __ldcs(y4 + i);
      float4 r;
      r.x = f(a.x, b.x);
      r.y = f(a.y, b.y);
      r.z = f(a.z, b.z);
      r.w = f(a.w, b.w);
      __stcs(o4 + i, r);
    }
    size_t rem = n & 3;
    if (tid < rem) out[n - rem + tid] = f(x[n - rem + tid], y[n - rem + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) out[i] = f(x[i], y[i]);
  }
}
// one input, two outputs (sincos): the functor's dual(x, out1, out2)
template <class F, bool VEC>
__global__ void __launch_bounds__(kBlock) k_dual32(const float *x, float *o1, float *o2, size_t n) {
  F f;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    size_t nq = n >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float4 *a4 = reinterpret_cast<float4 *>(o1);
    float4 *b4 = reinterpret_cast<float4 *>(o2);
    for (size_t i = tid; i < nq; i += stride) {
      float4 v = __ldcs(x4 + i), a, b;
      f.dual(v.x, a.x, b.x);
      f.dual(v.y, a.y, b.y);
      f.dual(v.z, a.z, b.z);
      f.dual(v.w, a.w, b.w);
      __stcs(a4 + i, a);
      __stcs(b4 + i, b);
    }
    size_t rem = n & 3;
    if (tid < rem) f.dual(x[n - rem + tid], o1[n - rem + tid], o2[n - rem + tid]);
  } else {
    for (size_t i = tid; i < n; i += stride) f.dual(x[i], o1[i], o2[i]);
  }
}
template <class F>
__global__ void __launch_bounds__(kBlock) k_sorted32(const float *x, float *out, size_t n) {
  constexpr int NC = F::NCLS, EPT = sort_ept<F>::value, TILE = kBlock * EPT;
  __shared__ float sx[TILE];                   // arguments, then results in place
  __shared__ unsigned short sidx[TILE];
  __shared__ int cnt[NC], cur[NC];
  F f;
  const int tid = threadIdx.x;
  const size_t ntiles = (n + TILE - 1) / TILE;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t base = tile * TILE;
    const int valid = (int)((n - base) < (size_t)TILE ? (n - base) : (size_t)TILE);
    if (tid < NC) cnt[tid] = 0;
    __syncthreads();
    int cl[EPT];
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      float v = 0.0f;
      cl[j] = -1;
      if (e < valid) {
        v = __ldcs(x + base + e);
        cl[j] = F::cls(v);
      }
      sx[e] = v;
    }
    sort_count<NC, EPT>(cl, cnt, tid);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int c = 0; c < NC; c++) { cur[c] = acc; acc += cnt[c]; }
    }
    __syncthreads();
    sort_scatter<NC, EPT>(cl, cur, sidx, tid);
    __syncthreads();
    for (int k = tid; k < valid; k += kBlock) {
      int e = sidx[k];
      sx[e] = f(sx[e]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EPT; j++) {
      int e = j * kBlock + tid;
      if (e < valid) __stcs(out + base + e, sx[e]);
    }
    __syncthreads();
  }
}

// Binary32 kernel with a deferred rare path.  A functor that declares
// DEFER has one expensive path that ordinary data takes rarely (the
// Payne-Hanek reduction of the trigonometric functions); in a plain kernel
// every warp holding one such lane runs that path with the others idle.
// Here the main pass evaluates every lane on one path: a lane with
// F::defer(x) runs on the stand-in argument F::kStandIn (a main-path value)
// and its true argument and position go to a shared-memory queue (one
// ballot and one atomic per warp); after a barrier the block evaluates the
// queue densely and overwrites those outputs.  Each output is still F(x) of
// its own argument, so results do not depend on the grouping.  Blocks take
// chunks of kDeferChunk elements (two 16-byte vectors per thread).
constexpr int kDeferVec = 2;
constexpr int kDeferChunk = kBlock * 4 * kDeferVec;

template <class F, class = void>
struct has_defer : std::false_type {};
template <class F>
struct has_defer<F, std::void_t<decltype(F::DEFER)>> : std::bool_constant<F::DEFER> {};

template <class F, int NOUT>
__device__ __forceinline__ void defer_eval(const F &f, float v, float &a, float &b) {
  if constexpr (NOUT == 1) {
    a = f(v);
    (void)b;
  } else {
    f.dual(v, a, b);
  }
}

template <class F, int NOUT>
__global__ void __launch_bounds__(kBlock) k_defer32(const float *x, float *o1, float *o2, size_t n) {
  __shared__ float qx[kDeferChunk];
  __shared__ unsigned short qi[kDeferChunk];
  __shared__ int qn;
  F f;
  const int tid = threadIdx.x;
  const unsigned lane = tid & 31, lt = (1u << lane) - 1u;
  const size_t nq = n >> 2;
  const size_t per = (size_t)kBlock * kDeferVec;
  const size_t nchunks = (nq + per - 1) / per;
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
  float4 *a4 = reinterpret_cast<float4 *>(o1);
  float4 *b4 = reinterpret_cast<float4 *>(o2);
  for (size_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    if (tid == 0) qn = 0;
    __syncthreads();
    const size_t q0 = c * per;
#pragma unroll 1
    for (int v = 0; v < kDeferVec; v++) {
      const int local = v * kBlock + tid;               // 16-byte vector within the chunk
      const size_t qv = q0 + local;
      const bool in = qv < nq;
      float4 t = in ? __ldcs(x4 + qv) : make_float4(0.f, 0.f, 0.f, 0.f);
      float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const bool r = in && F::defer(e[k]);
        const unsigned m = __ballot_sync(0xffffffffu, r);
        if (m) {
          const int leader = __ffs(m) - 1;
          int b = 0;
          if ((int)lane == leader) b = atomicAdd(&qn, __popc(m));
          b = __shfl_sync(0xffffffffu, b, leader);
          if (r) {
            qx[b + __popc(m & lt)] = e[k];
            qi[b + __popc(m & lt)] = (unsigned short)(local * 4 + k);
          }
        }
        if (r) e[k] = F::kStandIn;
      }
      float4 ra, rb;
      defer_eval<F, NOUT>(f, e[0], ra.x, rb.x);
      defer_eval<F, NOUT>(f, e[1], ra.y, rb.y);
      defer_eval<F, NOUT>(f, e[2], ra.z, rb.z);
      defer_eval<F, NOUT>(f, e[3], ra.w, rb.w);
      if (in) {
        __stcs(a4 + qv, ra);
        if constexpr (NOUT == 2) __stcs(b4 + qv, rb);
      }
    }
    __syncthreads();
    const int m = qn;
    for (int k = tid; k < m; k += kBlock) {
      const size_t g = q0 * 4 + qi[k];
      float a, b;
      defer_eval<F, NOUT>(f, qx[k], a, b);
      o1[g] = a;
      if constexpr (NOUT == 2) o2[g] = b;
    }
    __syncthreads();
  }
  const size_t rem = n & 3;
  if (blockIdx.x == 0 && (size_t)tid < rem) {
    const size_t g = n - rem + tid;
    float a, b;
    defer_eval<F, NOUT>(f, x[g], a, b);
    o1[g] = a;
    if constexpr (NOUT == 2) o2[g] = b;
  }
}

template <class F>
sleefcu_status launch_unary32(const char *name, const float *x, float *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if constexpr (has_defer<F>::value) {
    if (aligned16(x) && aligned16(out)) {
      auto k = k_defer32<F, 1>;
      k<<<grid_for((const void *)k, (n + 3) / 4 / kDeferVec), kBlock, 0, st>>>(x, out, out, n);
      return check_launch(name);
    }
  }
  if (aligned16(x) && aligned16(out)) {
    auto k = k_unary32<F, true>;
    k<<<grid_for((const void *)k, (n + 3) / 4), kBlock, 0, st>>>(x, out, n);
  } else {
    auto k = k_unary32<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, out, n);
  }
  return check_launch(name);
}
template <class F>
sleefcu_status launch_sorted32(const char *name, const float *x, float *out, size_t n, sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, out)) return rc_;
  auto k = k_sorted32<F>;
  constexpr int EPT = sort_ept<F>::value;
  k<<<grid_for((const void *)k, (n + EPT - 1) / EPT), kBlock, 0, (cudaStream_t)s>>>(x, out, n);
  return check_launch(name);
}

template <class F>
sleefcu_status launch_binary32(const char *name, const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !y || !out) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, y, out)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if (aligned16(x) && aligned16(y) && aligned16(out)) {
    auto k = k_binary32<F, true>;
    k<<<grid_for((const void *)k, (n + 3) / 4), kBlock, 0, st>>>(x, y, out, n);
  } else {
    auto k = k_binary32<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, y, out, n);
  }
  return check_launch(name);
}
template <class F>
sleefcu_status launch_dual32(const char *name, const float *x, float *o1, float *o2, size_t n,
                             sleefcu_stream s) {
  if (n == 0) return SLEEFCU_OK;
  if (!x || !o1 || !o2) { set_error("%s: null pointer with n = %zu", name, n); return SLEEFCU_EINVAL; }
  if (sleefcu_status rc_ = check_args(name, n, x, o1, o2)) return rc_;
  cudaStream_t st = (cudaStream_t)s;
  if constexpr (has_defer<F>::value) {
    if (aligned16(x) && aligned16(o1) && aligned16(o2)) {
      auto k = k_defer32<F, 2>;
      k<<<grid_for((const void *)k, (n + 3) / 4 / kDeferVec), kBlock, 0, st>>>(x, o1, o2, n);
      return check_launch(name);
    }
  }
  if (aligned16(x) && aligned16(o1) && aligned16(o2)) {
    auto k = k_dual32<F, true>;
    k<<<grid_for((const void *)k, (n + 3) / 4), kBlock, 0, st>>>(x, o1, o2, n);
  } else {
    auto k = k_dual32<F, false>;
    k<<<grid_for((const void *)k, n), kBlock, 0, st>>>(x, o1, o2, n);
  }
  return check_launch(name);
}

}  // namespace sleefcu
