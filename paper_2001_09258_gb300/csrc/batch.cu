// Batched mixed launch: many arrays of uneven length and mixed functions in
// one persistent kernel.
//
// A plan holds one descriptor per array (entry point code, pointers, n) and
// the prefix sums of each array's tile count.  The kernel runs one CTA per
// resident slot; CTAs claim tiles from a device counter, find the array of a
// tile by binary search over the prefix sums, and evaluate its elements with
// the same device functors as the individual entry points (so every output is
// bit-identical to the single-array call).  The switch over entry points is
// uniform within a CTA.  Block size, tile size (elements per thread x block
// size), vector width and grid multiplier are runtime parameters chosen by
// sleefcu_batch_autotune, which times candidate configurations on the plan
// itself and can cache the choice in a JSON file keyed by device name.
// The batched kernel runs multiplications and roundings in software through
// one out-of-line copy of the exact multiply (SLEEFCU_SOFT_MUL 2): measured
// on the 4096-array mix, 17.9 Gelem/s against 15.8 with the FP64 pipe's
// multiply and 15.1 with the software multiply inlined (its one kernel holds
// every functor, and the inlined copies cost more instruction fetch than
// they save).  The results are the same bits.
#define SLEEFCU_SOFT_MUL 2
#define SLEEFCU_FUNCTORS_ONLY
#include "trig_f64.cu"
#include "explog_f64.cu"
#include "pow_f64.cu"
#include "invtrig_f64.cu"
#include "fmod_f64.cu"
#include "trig_f32.cu"
#include "explog_f32.cu"
#include "derived_f64.cu"
#include "gamma_f64.cu"
#include "derived_f32.cu"
#undef SLEEFCU_FUNCTORS_ONLY

#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <type_traits>
#include <vector>

namespace sleefcu {
namespace batch {

enum Kind { U64, B64, SC64, U32, B32, SC32, BF, HF };

// entry point table: code (= position), name, kind, functor
#define SLEEFCU_BATCH_TABLE(X) \
  X(0, "sin_u10_f64", U64, trig64::SinU10) \
  X(1, "sin_u35_f64", U64, trig64::SinU35) \
  X(2, "cos_u10_f64", U64, trig64::CosU10) \
  X(3, "cos_u35_f64", U64, trig64::CosU35) \
  X(4, "tan_u10_f64", U64, trig64::TanU10) \
  X(5, "tan_u35_f64", U64, trig64::TanU35) \
  X(6, "sincos_u10_f64", SC64, trig64::SinCosU10) \
  X(7, "sincos_u35_f64", SC64, trig64::SinCosU35) \
  X(8, "asin_u10_f64", U64, invtrig64::AsinU10) \
  X(9, "asin_u35_f64", U64, invtrig64::AsinU35) \
  X(10, "acos_u10_f64", U64, invtrig64::AcosU10) \
  X(11, "acos_u35_f64", U64, invtrig64::AcosU35) \
  X(12, "atan_u10_f64", U64, invtrig64::AtanU10) \
  X(13, "atan_u35_f64", U64, invtrig64::AtanU35) \
  X(14, "atan2_u10_f64", B64, invtrig64::Atan2U10) \
  X(15, "atan2_u35_f64", B64, invtrig64::Atan2U35) \
  X(16, "exp_u10_f64", U64, explog64::ExpU10) \
  X(17, "exp_u35_f64", U64, explog64::ExpU35) \
  X(18, "log_u10_f64", U64, explog64::LogU10) \
  X(19, "log_u35_f64", U64, explog64::LogU35) \
  X(20, "pow_u10_f64", B64, explog64::PowU10) \
  X(21, "pow_u35_f64", B64, explog64::PowU10) \
  X(22, "fmod_u10_f64", B64, fmod64::FmodF) \
  X(23, "fmod_u35_f64", B64, fmod64::FmodF) \
  X(24, "remainder_u10_f64", B64, fmod64::RemainderF) \
  X(25, "remainder_u35_f64", B64, fmod64::RemainderF) \
  X(26, "sin_u10_f32", U32, trig32::SinU10) \
  X(27, "sin_u35_f32", U32, trig32::SinU35) \
  X(28, "cos_u10_f32", U32, trig32::CosU10) \
  X(29, "cos_u35_f32", U32, trig32::CosU35) \
  X(30, "exp_u10_f32", U32, explog32::ExpU10) \
  X(31, "exp_u35_f32", U32, explog32::ExpU35) \
  X(32, "log_u10_f32", U32, explog32::LogU10) \
  X(33, "log_u35_f32", U32, explog32::LogU35) \
  X(34, "log1p_u10_f32", U32, explog32::Log1pU10) \
  X(35, "log1p_u35_f32", U32, explog32::Log1pU35) \
  X(36, "tanh_u10_f32", U32, explog32::TanhU10) \
  X(37, "tanh_u35_f32", U32, explog32::TanhU35) \
  X(38, "erf_u10_f32", U32, explog32::ErfU10) \
  X(39, "erf_u35_f32", U32, explog32::ErfU35) \
  X(40, "erf_u10_bf16", BF, explog32::ErfU10) \
  X(41, "erf_u35_bf16", BF, explog32::ErfU35) \
  X(42, "tanh_u10_bf16", BF, explog32::TanhU10) \
  X(43, "tanh_u35_bf16", BF, explog32::TanhU35) \
  X(44, "exp_u10_bf16", BF, explog32::ExpU10) \
  X(45, "exp_u35_bf16", BF, explog32::ExpU35) \
  X(46, "log1p_u10_bf16", BF, explog32::Log1pU10) \
  X(47, "log1p_u35_bf16", BF, explog32::Log1pU35) \
  X(48, "erf_u10_f16", HF, explog32::ErfU10) \
  X(49, "erf_u35_f16", HF, explog32::ErfU35) \
  X(50, "tanh_u10_f16", HF, explog32::TanhU10) \
  X(51, "tanh_u35_f16", HF, explog32::TanhU35) \
  X(52, "exp_u10_f16", HF, explog32::ExpU10) \
  X(53, "exp_u35_f16", HF, explog32::ExpU35) \
  X(54, "log1p_u10_f16", HF, explog32::Log1pU10) \
  X(55, "log1p_u35_f16", HF, explog32::Log1pU35) \
  X(56, "exp2_u10_f64", U64, derived64::Exp2U10) \
  X(57, "exp2_u35_f64", U64, derived64::Exp2U35) \
  X(58, "exp10_u10_f64", U64, derived64::Exp10U10) \
  X(59, "exp10_u35_f64", U64, derived64::Exp10U35) \
  X(60, "expm1_u10_f64", U64, derived64::Expm1U10) \
  X(61, "expm1_u35_f64", U64, derived64::Expm1U35) \
  X(62, "log2_u10_f64", U64, derived64::Log2U10) \
  X(63, "log2_u35_f64", U64, derived64::Log2U35) \
  X(64, "log10_u10_f64", U64, derived64::Log10U10) \
  X(65, "log10_u35_f64", U64, derived64::Log10U35) \
  X(66, "log1p_u10_f64", U64, derived64::Log1pU10) \
  X(67, "log1p_u35_f64", U64, derived64::Log1pU35) \
  X(68, "cbrt_u10_f64", U64, derived64::CbrtU10) \
  X(69, "cbrt_u35_f64", U64, derived64::CbrtU35) \
  X(70, "sinh_u10_f64", U64, derived64::SinhU10) \
  X(71, "sinh_u35_f64", U64, derived64::SinhU35) \
  X(72, "cosh_u10_f64", U64, derived64::CoshU10) \
  X(73, "cosh_u35_f64", U64, derived64::CoshU35) \
  X(74, "tanh_u10_f64", U64, derived64::TanhU10) \
  X(75, "tanh_u35_f64", U64, derived64::TanhU35) \
  X(76, "asinh_u10_f64", U64, derived64::AsinhU10) \
  X(77, "asinh_u35_f64", U64, derived64::AsinhU35) \
  X(78, "acosh_u10_f64", U64, derived64::AcoshU10) \
  X(79, "acosh_u35_f64", U64, derived64::AcoshU35) \
  X(80, "atanh_u10_f64", U64, derived64::AtanhU10) \
  X(81, "atanh_u35_f64", U64, derived64::AtanhU35) \
  X(82, "erf_u10_f64", U64, derived64::ErfU10) \
  X(83, "erf_u35_f64", U64, derived64::ErfU35) \
  X(84, "erfc_u10_f64", U64, derived64::ErfcU10) \
  X(85, "erfc_u35_f64", U64, derived64::ErfcU10) \
  X(86, "tgamma_u10_f64", U64, gamma64::TgammaU10) \
  X(87, "tgamma_u35_f64", U64, gamma64::TgammaU10) \
  X(88, "lgamma_u10_f64", U64, gamma64::LgammaU10) \
  X(89, "lgamma_u35_f64", U64, gamma64::LgammaU10) \
  X(90, "tan_u10_f32", U32, derived32::TanU10) \
  X(91, "tan_u35_f32", U32, derived32::TanU35) \
  X(92, "sincos_u10_f32", SC32, derived32::SinCosU10) \
  X(93, "sincos_u35_f32", SC32, derived32::SinCosU35) \
  X(94, "asin_u10_f32", U32, derived32::AsinU10) \
  X(95, "asin_u35_f32", U32, derived32::AsinU35) \
  X(96, "acos_u10_f32", U32, derived32::AcosU10) \
  X(97, "acos_u35_f32", U32, derived32::AcosU35) \
  X(98, "atan_u10_f32", U32, derived32::AtanU10) \
  X(99, "atan_u35_f32", U32, derived32::AtanU35) \
  X(100, "atan2_u10_f32", B32, derived32::Atan2U10) \
  X(101, "atan2_u35_f32", B32, derived32::Atan2U35) \
  X(102, "exp2_u10_f32", U32, derived32::Exp2U10) \
  X(103, "exp2_u35_f32", U32, derived32::Exp2U35) \
  X(104, "exp10_u10_f32", U32, derived32::Exp10U10) \
  X(105, "exp10_u35_f32", U32, derived32::Exp10U35) \
  X(106, "expm1_u10_f32", U32, derived32::Expm1U10) \
  X(107, "expm1_u35_f32", U32, derived32::Expm1U10) \
  X(108, "log2_u10_f32", U32, derived32::Log2U10) \
  X(109, "log2_u35_f32", U32, derived32::Log2U35) \
  X(110, "log10_u10_f32", U32, derived32::Log10U10) \
  X(111, "log10_u35_f32", U32, derived32::Log10U35) \
  X(112, "pow_u10_f32", B32, derived32::PowU10) \
  X(113, "pow_u35_f32", B32, derived32::PowU10) \
  X(114, "cbrt_u10_f32", U32, derived32::CbrtU10) \
  X(115, "cbrt_u35_f32", U32, derived32::CbrtU35) \
  X(116, "sinh_u10_f32", U32, derived32::SinhU10) \
  X(117, "sinh_u35_f32", U32, derived32::SinhU10) \
  X(118, "cosh_u10_f32", U32, derived32::CoshU10) \
  X(119, "cosh_u35_f32", U32, derived32::CoshU10) \
  X(120, "asinh_u10_f32", U32, derived32::AsinhU10) \
  X(121, "asinh_u35_f32", U32, derived32::AsinhU35) \
  X(122, "acosh_u10_f32", U32, derived32::AcoshU10) \
  X(123, "acosh_u35_f32", U32, derived32::AcoshU35) \
  X(124, "atanh_u10_f32", U32, derived32::AtanhU10) \
  X(125, "atanh_u35_f32", U32, derived32::AtanhU35) \
  X(126, "erfc_u10_f32", U32, derived32::ErfcU10) \
  X(127, "erfc_u35_f32", U32, derived32::ErfcU10) \
  X(128, "fmod_u10_f32", B32, derived32::FmodF) \
  X(129, "fmod_u35_f32", B32, derived32::FmodF) \
  X(130, "remainder_u10_f32", B32, derived32::RemainderF) \
  X(131, "remainder_u35_f32", B32, derived32::RemainderF) \
  X(132, "tgamma_u10_f32", U32, derived32::TgammaU10) \
  X(133, "tgamma_u35_f32", U32, derived32::TgammaU10) \
  X(134, "lgamma_u10_f32", U32, derived32::LgammaU10) \
  X(135, "lgamma_u35_f32", U32, derived32::LgammaU10)

#define SLEEFCU_BATCH_NAME(c, name, kind, F) name,
static const char *kNames[] = {SLEEFCU_BATCH_TABLE(SLEEFCU_BATCH_NAME)};
#undef SLEEFCU_BATCH_NAME
constexpr int kCodes = sizeof(kNames) / sizeof(kNames[0]);

struct Desc {
  const void *x, *y;
  void *out, *out2;
  long long n;
  int code, pad;
};

// functors with several reduction paths expose NCLS and cls(); their tiles
// are evaluated in divergence-sorted sub-tiles (the single-array sorted
// kernels' scheme, for any block size 128..512)
template <class F, class = void> struct sortable { static constexpr bool value = false; };
template <class F> struct sortable<F, decltype((void)F::NCLS)> { static constexpr bool value = true; };

template <class F, class = void> struct sort_f32 { static constexpr bool value = false; };
template <class F> struct sort_f32<F, decltype((void)F::SORT32)> { static constexpr bool value = F::SORT32; };

constexpr int kSubTile = 1024;         // elements per sorted sub-tile
constexpr int kMaxEPT = 8;             // kSubTile / smallest block size
struct SortSmem {
  double x[kSubTile], y[kSubTile];     // inputs, then results (in place)
  unsigned short idx[kSubTile];
  int cnt[64], cur[64];
};

template <Kind K, class F>
__device__ __forceinline__ void run_sorted(const Desc &D, long long b, long long e, SortSmem &S) {
  using T = typename std::conditional<(K == U64 || K == B64 || K == SC64), double, float>::type;
  constexpr bool BIN = (K == B64 || K == B32), DUAL = (K == SC64 || K == SC32);
  F f;
  const T *x = (const T *)D.x, *y = (const T *)D.y;
  T *o = (T *)D.out, *o2 = (T *)D.out2;
  T *sx = (T *)S.x, *sy = (T *)S.y;
  const int tid = threadIdx.x, nt = blockDim.x, ept = kSubTile / nt;
  const unsigned lane = tid & 31, lt = (1u << lane) - 1u;
  for (long long base = b; base < e; base += kSubTile) {
    const int valid = (int)(e - base < kSubTile ? e - base : kSubTile);
    if (tid < F::NCLS) S.cnt[tid] = 0;
    __syncthreads();
    int cl[kMaxEPT];
#pragma unroll
    for (int j = 0; j < kMaxEPT; j++) {
      cl[j] = -1;
      if (j < ept) {
        int el = j * nt + tid;
        T a = 0, c = 0;
        if (el < valid) {
          a = x[base + el];
          if constexpr (BIN) {
            c = y[base + el];
            cl[j] = F::cls(a, c);
          } else {
            cl[j] = F::cls(a);
          }
        }
        sx[el] = a;
        if constexpr (BIN) sy[el] = c;
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxEPT; j++) {
      if (j < ept) {
        unsigned m = __match_any_sync(0xffffffffu, cl[j]);
        if ((int)lane == __ffs(m) - 1 && cl[j] >= 0) atomicAdd(&S.cnt[cl[j]], __popc(m));
      }
    }
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int c = 0; c < F::NCLS; c++) { S.cur[c] = acc; acc += S.cnt[c]; }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kMaxEPT; j++) {
      if (j < ept) {
        unsigned m = __match_any_sync(0xffffffffu, cl[j]);
        int leader = __ffs(m) - 1, p = 0;
        if ((int)lane == leader && cl[j] >= 0) p = atomicAdd(&S.cur[cl[j]], __popc(m));
        p = __shfl_sync(0xffffffffu, p, leader);
        if (cl[j] >= 0) S.idx[p + __popc(m & lt)] = (unsigned short)(j * nt + tid);
      }
    }
    __syncthreads();
    for (int k = tid; k < valid; k += nt) {
      int el = S.idx[k];
      if constexpr (DUAL) {
        T a, c;
        f.dual(sx[el], a, c);
        sx[el] = a;
        sy[el] = c;
      } else if constexpr (BIN) {
        sx[el] = f(sx[el], sy[el]);
      } else {
        sx[el] = f(sx[el]);
      }
    }
    __syncthreads();
    for (int el = tid; el < valid; el += nt) {
      o[base + el] = sx[el];
      if constexpr (DUAL) o2[base + el] = sy[el];
    }
    __syncthreads();
  }
}

// binary32 functors with a deferred rare path (DEFER, as in k_defer32): per
// sub-tile, every lane runs the main path (deferred lanes on the stand-in
// argument), the deferred arguments are queued in shared memory and, after a
// barrier, evaluated densely and written over the stand-in results
template <Kind K, class F>
__device__ __forceinline__ void run_deferred(const Desc &D, long long b, long long e, SortSmem &S) {
  constexpr bool DUAL = (K == SC32);
  F f;
  const float *x = (const float *)D.x;
  float *o = (float *)D.out, *o2 = (float *)D.out2;
  float *qx = (float *)S.x;
  const int tid = threadIdx.x, nt = blockDim.x, ept = kSubTile / nt;
  const unsigned lane = tid & 31, lt = (1u << lane) - 1u;
  for (long long base = b; base < e; base += kSubTile) {
    const int valid = (int)(e - base < kSubTile ? e - base : kSubTile);
    if (tid == 0) S.cnt[0] = 0;
    __syncthreads();
#pragma unroll 1
    for (int j = 0; j < ept; j++) {
      const int el = j * nt + tid;
      const bool in = el < valid;
      float v = in ? x[base + el] : 0.0f;
      const bool r = in && F::defer(v);
      const unsigned m = __ballot_sync(0xffffffffu, r);
      if (m) {
        const int leader = __ffs(m) - 1;
        int p = 0;
        if ((int)lane == leader) p = atomicAdd(&S.cnt[0], __popc(m));
        p = __shfl_sync(0xffffffffu, p, leader);
        if (r) {
          qx[p + __popc(m & lt)] = v;
          S.idx[p + __popc(m & lt)] = (unsigned short)el;
        }
      }
      if (r) v = F::kStandIn;
      if constexpr (DUAL) {
        float a, c;
        f.dual(v, a, c);
        if (in) {
          o[base + el] = a;
          o2[base + el] = c;
        }
      } else {
        const float a = f(v);
        if (in) o[base + el] = a;
      }
    }
    __syncthreads();
    const int q = S.cnt[0];
    for (int k = tid; k < q; k += nt) {
      const long long g = base + S.idx[k];
      if constexpr (DUAL) {
        f.dual(qx[k], o[g], o2[g]);
      } else {
        o[g] = f(qx[k]);
      }
    }
    __syncthreads();
  }
}

// evaluate elements [b, e) of one array; threads of the CTA stride over them,
// vec > 1 uses 16-byte accesses when the tile start is aligned
template <Kind K, class F>
__device__ __forceinline__ void run(const Desc &D, long long b, long long e, int vec, SortSmem &S) {
  if constexpr ((K == U32 || K == SC32) && has_defer<F>::value) {
    if (kSubTile % blockDim.x == 0 && kSubTile / blockDim.x <= kMaxEPT) {   // blocks of 128..1024 threads
      run_deferred<K, F>(D, b, e, S);
      return;
    }
  }
  // FP64 functors with several paths always; binary32 ones only where the
  // paths differ by an order of magnitude (gamma's eight classes)
  if constexpr (sortable<F>::value && K != BF && K != HF &&
                (K == U64 || K == B64 || K == SC64 || sort_f32<F>::value)) {
    if (kSubTile % blockDim.x == 0 && kSubTile / blockDim.x <= kMaxEPT) {   // blocks of 128..1024 threads
      run_sorted<K, F>(D, b, e, S);
      return;
    }
  }
  F f;
  const int tid = threadIdx.x, nt = blockDim.x;
  if constexpr (K == U64) {
    const double *x = (const double *)D.x;
    double *o = (double *)D.out;
    if (vec > 1 && ((((uintptr_t)(x + b)) | ((uintptr_t)(o + b))) & 15) == 0) {
      long long np = (e - b) >> 1;
      for (long long i = tid; i < np; i += nt) {
        double2 v = __ldcs(reinterpret_cast<const double2 *>(x + b) + i), r;
        r.x = f(v.x);
        r.y = f(v.y);
        __stcs(reinterpret_cast<double2 *>(o + b) + i, r);
      }
      if (((e - b) & 1) && tid == 0) o[e - 1] = f(x[e - 1]);
    } else {
      for (long long i = b + tid; i < e; i += nt) o[i] = f(x[i]);
    }
  } else if constexpr (K == B64) {
    const double *x = (const double *)D.x, *y = (const double *)D.y;
    double *o = (double *)D.out;
    for (long long i = b + tid; i < e; i += nt) o[i] = f(x[i], y[i]);
  } else if constexpr (K == SC64) {
    const double *x = (const double *)D.x;
    double *o = (double *)D.out, *o2 = (double *)D.out2;
    for (long long i = b + tid; i < e; i += nt) f.dual(x[i], o[i], o2[i]);
  } else if constexpr (K == U32) {
    const float *x = (const float *)D.x;
    float *o = (float *)D.out;
    if (vec > 1 && ((((uintptr_t)(x + b)) | ((uintptr_t)(o + b))) & 15) == 0) {
      long long nq = (e - b) >> 2;
      for (long long i = tid; i < nq; i += nt) {
        float4 v = __ldcs(reinterpret_cast<const float4 *>(x + b) + i), r;
        r.x = f(v.x);
        r.y = f(v.y);
        r.z = f(v.z);
        r.w = f(v.w);
        __stcs(reinterpret_cast<float4 *>(o + b) + i, r);
      }
      for (long long i = b + 4 * nq + tid; i < e; i += nt) o[i] = f(x[i]);
    } else {
      for (long long i = b + tid; i < e; i += nt) o[i] = f(x[i]);
    }
  } else if constexpr (K == B32) {
    const float *x = (const float *)D.x, *y = (const float *)D.y;
    float *o = (float *)D.out;
    for (long long i = b + tid; i < e; i += nt) o[i] = f(x[i], y[i]);
  } else if constexpr (K == SC32) {
    const float *x = (const float *)D.x;
    float *o = (float *)D.out, *o2 = (float *)D.out2;
    for (long long i = b + tid; i < e; i += nt) f.dual(x[i], o[i], o2[i]);
  } else {
    const uint16_t *x = (const uint16_t *)D.x;
    uint16_t *o = (uint16_t *)D.out;
    for (long long i = b + tid; i < e; i += nt) o[i] = lowp::ev<F, K == BF>(f, x[i]);
  }
}

__global__ void __launch_bounds__(512) k_batch(const Desc *__restrict__ d, const long long *__restrict__ pre,
                                               int nitems, long long ntiles, int tile, int vec,
                                               unsigned long long *ctr) {
  __shared__ long long s_t;
  __shared__ int s_i;
  __shared__ SortSmem S;
  for (;;) {
    if (threadIdx.x == 0) {
      long long t = (long long)atomicAdd(ctr, 1ull);
      int lo = 0, hi = nitems - 1;          // last item with pre[item] <= t
      if (t < ntiles) {
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
      }
      s_t = t;
      s_i = lo;
    }
    __syncthreads();
    long long t = s_t;
    int item = s_i;
    __syncthreads();
    if (t >= ntiles) break;
    Desc D = d[item];
    long long b = (t - pre[item]) * (long long)tile;
    long long e = b + tile < D.n ? b + tile : D.n;
    switch (D.code) {
#define SLEEFCU_BATCH_CASE(c, name, kind, F) \
  case c: run<kind, F>(D, b, e, vec, S); break;
      SLEEFCU_BATCH_TABLE(SLEEFCU_BATCH_CASE)
#undef SLEEFCU_BATCH_CASE
      default: break;
    }
  }
}

}  // namespace batch
}  // namespace sleefcu

// ---------------- host side ----------------
namespace {
using namespace sleefcu;
using namespace sleefcu::batch;

const char *kFnNames[SLEEFCU_FN_COUNT] = {"sin",   "cos",   "tan",   "sincos", "asin",  "acos",  "atan",
                                          "atan2", "exp",   "log",   "pow",    "fmod",  "remainder",
                                          "log1p", "tanh",  "erf",   "exp2",   "exp10", "expm1", "log2",
                                          "log10", "cbrt",  "sinh",  "cosh",   "asinh", "acosh", "atanh",
                                          "erfc",  "tgamma", "lgamma"};
const char *kTypeNames[4] = {"f64", "f32", "bf16", "f16"};

// (fn, dtype, ulp) -> entry point code, and the operands each code needs:
// tables built once from the entry point names, so that a lookup is one load
struct CodeTables {
  short code[SLEEFCU_FN_COUNT][4][2];
  bool y[kCodes], out2[kCodes];
  CodeTables() {
    for (int f = 0; f < SLEEFCU_FN_COUNT; f++)
      for (int t = 0; t < 4; t++)
        for (int u = 0; u < 2; u++) {
          char name[64];
          snprintf(name, sizeof name, "%s_u%d_%s", kFnNames[f], u ? 35 : 10, kTypeNames[t]);
          code[f][t][u] = -1;
          for (int c = 0; c < kCodes; c++)
            if (!strcmp(kNames[c], name)) code[f][t][u] = (short)c;
        }
    for (int c = 0; c < kCodes; c++) {
      y[c] = strstr(kNames[c], "atan2_") || strstr(kNames[c], "pow_") || strstr(kNames[c], "fmod_") ||
             strstr(kNames[c], "remainder_");
      out2[c] = strstr(kNames[c], "sincos_") != nullptr;
    }
  }
};
const CodeTables &code_tables() {
  static const CodeTables t;           // thread-safe one-time initialization
  return t;
}
int code_of(const sleefcu_batch_item &it) {
  if (it.fn >= SLEEFCU_FN_COUNT || it.dtype > 3 || (it.ulp != 10 && it.ulp != 35)) return -1;
  return code_tables().code[it.fn][it.dtype][it.ulp == 35];
}
bool needs_y(int code) { return code_tables().y[code]; }
bool needs_out2(int code) { return code_tables().out2[code]; }
}  // namespace

struct sleefcu_batch {
  int dev = 0, sms = 0;
  std::vector<Desc> desc;              // non-empty items only
  Desc *d_desc = nullptr;
  long long *d_pre = nullptr;
  unsigned long long *d_ctr = nullptr;
  long long ntiles = 0;
  int block = 256, tile = 4096, grid_mult = 2, vec = 2;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void drop_graph(sleefcu_batch *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

// tile prefix sums for the current tile size (synchronous upload)
static sleefcu_status upload_prefix(sleefcu_batch *p) {
  std::vector<long long> pre(p->desc.size() + 1, 0);
  for (size_t i = 0; i < p->desc.size(); i++) pre[i + 1] = pre[i] + (p->desc[i].n + p->tile - 1) / p->tile;
  p->ntiles = pre.back();
  if (p->desc.empty()) return SLEEFCU_OK;
  cudaError_t e = cudaMemcpy(p->d_pre, pre.data(), pre.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { set_error("sleefcu_batch: %s", cudaGetErrorString(e)); return SLEEFCU_ECUDA; }
  return SLEEFCU_OK;
}

// checked build: every array of an item must be device memory holding its n elements
static sleefcu_status check_item(const char *name, const sleefcu_batch_item &it, int code) {
  size_t es = it.dtype == SLEEFCU_F64 ? 8 : it.dtype == SLEEFCU_F32 ? 4 : 2;
  if (sleefcu_status r = check_args(name, it.n * es, (const unsigned char *)it.x,
                                    (const unsigned char *)it.out))
    return r;
  if (needs_y(code))
    if (sleefcu_status r = check_args(name, it.n * es, (const unsigned char *)it.y)) return r;
  if (needs_out2(code))
    if (sleefcu_status r = check_args(name, it.n * es, (const unsigned char *)it.out2)) return r;
  return SLEEFCU_OK;
}

extern "C" sleefcu_status sleefcu_batch_create(const sleefcu_batch_item *items, size_t count,
                                               const char *tune_file_or_null, sleefcu_batch **plan) {
  if (!plan || (count && !items)) { set_error("sleefcu_batch_create: null argument"); return SLEEFCU_EINVAL; }
  *plan = nullptr;
  sleefcu_batch *p = new sleefcu_batch();
  for (size_t i = 0; i < count; i++) {
    const sleefcu_batch_item &it = items[i];
    int c = code_of(it);
    if (c < 0) {
      set_error("sleefcu_batch_create: item %zu: unsupported (fn %u, dtype %u, ulp %u)", i, it.fn, it.dtype, it.ulp);
      delete p;
      return SLEEFCU_EUNSUPPORTED;
    }
    if (it.n == 0) continue;
    if (!it.x || !it.out || (needs_y(c) && !it.y) || (needs_out2(c) && !it.out2)) {
      set_error("sleefcu_batch_create: item %zu: null pointer with n = %zu", i, it.n);
      delete p;
      return SLEEFCU_EINVAL;
    }
    if (sleefcu_status r = check_item("sleefcu_batch_create", it, c)) {
      delete p;
      return r;
    }
    p->desc.push_back(Desc{it.x, it.y, it.out, it.out2, (long long)it.n, c, 0});
  }
  cudaGetDevice(&p->dev);
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->dev);
  if (!p->desc.empty()) {
    size_t nd = p->desc.size();
    if (cudaMalloc(&p->d_desc, nd * sizeof(Desc)) != cudaSuccess ||
        cudaMalloc(&p->d_pre, (nd + 1) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&p->d_ctr, sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      set_error("sleefcu_batch_create: out of device memory");
      sleefcu_batch_destroy(p);
      return SLEEFCU_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(p->d_desc, p->desc.data(), nd * sizeof(Desc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_error("sleefcu_batch_create: %s", cudaGetErrorString(e));
      sleefcu_batch_destroy(p);
      return SLEEFCU_ECUDA;
    }
  }
  sleefcu_status st = upload_prefix(p);
  if (st == SLEEFCU_OK && tune_file_or_null)
    st = sleefcu_batch_autotune(p, *tune_file_or_null ? tune_file_or_null : nullptr, nullptr);
  if (st == SLEEFCU_OK && tune_file_or_null && cudaStreamSynchronize(nullptr) != cudaSuccess) {
    set_error("sleefcu_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
    st = SLEEFCU_ECUDA;
  }
  if (st != SLEEFCU_OK) { sleefcu_batch_destroy(p); return st; }
  *plan = p;
  return SLEEFCU_OK;
}

extern "C" void sleefcu_batch_destroy(sleefcu_batch *p) {
  if (!p) return;
  drop_graph(p);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->d_desc);
  cudaFree(p->d_pre);
  cudaFree(p->d_ctr);
  delete p;
}

static int batch_grid(sleefcu_batch *p) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_batch, p->block, 0);
  if (per < 1) per = 1;
  long long g = (long long)p->sms * per * p->grid_mult;
  if (g > p->ntiles) g = p->ntiles;
  return (int)(g < 1 ? 1 : g);
}

static sleefcu_status enqueue(sleefcu_batch *p, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p->d_ctr, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) { set_error("sleefcu_batch_launch: %s", cudaGetErrorString(e)); return SLEEFCU_ECUDA; }
  k_batch<<<batch_grid(p), p->block, 0, st>>>(p->d_desc, p->d_pre, (int)p->desc.size(), p->ntiles, p->tile,
                                               p->vec, p->d_ctr);
  return check_launch("sleefcu_batch_launch");
}

extern "C" sleefcu_status sleefcu_batch_launch(sleefcu_batch *p, sleefcu_stream s) {
  if (!p) { set_error("sleefcu_batch_launch: null plan"); return SLEEFCU_EINVAL; }
  if (p->ntiles == 0) return SLEEFCU_OK;
  return enqueue(p, (cudaStream_t)s);
}

extern "C" sleefcu_status sleefcu_batch_launch_graph(sleefcu_batch *p, sleefcu_stream s) {
  if (!p) { set_error("sleefcu_batch_launch_graph: null plan"); return SLEEFCU_EINVAL; }
  if (p->ntiles == 0) return SLEEFCU_OK;
  if (!p->exec) {
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("sleefcu_batch_launch_graph: cannot create the capture stream");
      return SLEEFCU_ECUDA;
    }
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { set_error("sleefcu_batch_launch_graph: %s", cudaGetErrorString(e)); return SLEEFCU_ECUDA; }
    sleefcu_status st = enqueue(p, p->cap);
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (st != SLEEFCU_OK) { drop_graph(p); return st; }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
      drop_graph(p);
      set_error("sleefcu_batch_launch_graph: %s", cudaGetErrorString(e));
      return SLEEFCU_ECUDA;
    }
  }
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)s);
  if (e != cudaSuccess) { set_error("sleefcu_batch_launch_graph: %s", cudaGetErrorString(e)); return SLEEFCU_ECUDA; }
  return SLEEFCU_OK;
}

extern "C" sleefcu_status sleefcu_batch_set_config(sleefcu_batch *p, int block, int tile, int grid_mult, int vec) {
  if (!p || block < 32 || block > 512 || (block & 31) || tile < block || grid_mult < 1 || grid_mult > 16 ||
      (vec != 1 && vec != 2)) {
    set_error("sleefcu_batch_set_config: bad argument");
    return SLEEFCU_EINVAL;
  }
  p->block = block;
  p->tile = tile;
  p->grid_mult = grid_mult;
  p->vec = vec;
  drop_graph(p);
  return upload_prefix(p);
}

extern "C" sleefcu_status sleefcu_batch_get_config(const sleefcu_batch *p, int *block, int *tile, int *grid_mult,
                                                   int *vec) {
  if (!p) { set_error("sleefcu_batch_get_config: null plan"); return SLEEFCU_EINVAL; }
  if (block) *block = p->block;
  if (tile) *tile = p->tile;
  if (grid_mult) *grid_mult = p->grid_mult;
  if (vec) *vec = p->vec;
  return SLEEFCU_OK;
}

// the plan's signature for the tuning cache: device name, array count, elements
static std::string signature(const sleefcu_batch *p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->dev);
  long long el = 0;
  for (const Desc &d : p->desc) el += d.n;
  char buf[512];
  snprintf(buf, sizeof buf, "%s|items=%zu|elems=%lld", prop.name, p->desc.size(), el);
  return buf;
}

extern "C" sleefcu_status sleefcu_batch_autotune(sleefcu_batch *p, const char *cache_file, sleefcu_stream s) {
  if (!p) { set_error("sleefcu_batch_autotune: null plan"); return SLEEFCU_EINVAL; }
  if (p->ntiles == 0) return SLEEFCU_OK;
  std::string sig = signature(p);
  if (cache_file) {                    // JSON lines: {"signature": "...", "block": b, "tile": t, ...}
    if (FILE *f = fopen(cache_file, "r")) {
      char line[1024];
      int b = 0, t = 0, g = 0, v = 0, found = 0;
      while (fgets(line, sizeof line, f)) {
        const char *k = strstr(line, "\"signature\": \"");
        if (!k || strncmp(k + 14, sig.c_str(), sig.size()) || k[14 + sig.size()] != '"') continue;
        const char *c = strstr(line, "\"block\":");
        if (c && sscanf(c, "\"block\": %d, \"tile\": %d, \"grid_mult\": %d, \"vec\": %d", &b, &t, &g, &v) == 4)
          found = 1;
      }
      fclose(f);
      if (found) return sleefcu_batch_set_config(p, b, t, g, v);
    }
  }
  cudaStream_t st = (cudaStream_t)s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks[] = {128, 256, 512};
  const int ept[] = {4, 16, 64};            // elements per thread: tile = ept x block
  const int mults[] = {1, 2, 4};
  const int vecs[] = {1, 2};
  float best = 1e30f;
  int bb = p->block, bt = p->tile, bg = p->grid_mult, bv = p->vec;
  for (int b : blocks)
    for (int e : ept)
      for (int g : mults)
        for (int v : vecs) {
          if (sleefcu_batch_set_config(p, b, e * b, g, v) != SLEEFCU_OK) continue;
          enqueue(p, st);                    // warm-up
          cudaEventRecord(e0, st);
          for (int r = 0; r < 3; r++) enqueue(p, st);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) { best = ms; bb = b; bt = e * b; bg = g; bv = v; }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  sleefcu_status rc = sleefcu_batch_set_config(p, bb, bt, bg, bv);
  if (rc == SLEEFCU_OK && cache_file) {
    if (FILE *f = fopen(cache_file, "a")) {
      fprintf(f, "{\"signature\": \"%s\", \"block\": %d, \"tile\": %d, \"grid_mult\": %d, \"vec\": %d, \"ms\": %.4f}\n",
              sig.c_str(), bb, bt, bg, bv, best / 3);
      fclose(f);
    }
  }
  return rc;
}

// ---------------- batched launch without allocation ----------------
// sleefcu_batch_create allocates device buffers for a plan.  Some callers
// cannot do that at the point where they launch: an embedding whose own
// caching allocator owns all of the device memory (a stray cudaMalloc
// fragments it or fails outright), or a latency-critical path where an
// allocation, and the device-wide synchronization that cudaFree implies,
// is not acceptable.  For them this entry point keeps the descriptors, the
// tile prefix sums and the tile counter in one fixed device array of file
// scope, sized for at most kStaticItems arrays (about 230 KB), and runs the
// same k_batch kernel with the default configuration.  The descriptors reach
// the array as arguments of small staging kernels (up to kStageItems per
// launch), not by copies from host memory: a copy from pageable host memory
// would first wait for all earlier work on the stream.
namespace {
constexpr size_t kStaticItems = 4096;
constexpr size_t kStaticDescBytes = kStaticItems * sizeof(sleefcu::batch::Desc);
constexpr size_t kStaticPreBytes = (kStaticItems + 1) * sizeof(long long);
constexpr size_t kStaticBytes = kStaticDescBytes + kStaticPreBytes + sizeof(unsigned long long);
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticBlock = 256, kStaticTile = 4096, kStaticGridMult = 2, kStaticVec = 2;
std::mutex g_static_mu;                                   // guards the address table
void *g_static_dev[kStaticMaxDevices];                     // scratch address per device
}  // namespace

namespace sleefcu {
namespace batch {
constexpr int kStageItems = 512;
// one staging launch: descriptors first .. first+count-1 and their prefix sums
struct StageChunk {
  Desc desc[kStageItems];
  long long pre[kStageItems];            // pre[j]: tiles of items 0 .. first+j
  int first, count;
};
static_assert(sizeof(StageChunk) < 32000, "staging chunk exceeds the kernel argument limit");
}  // namespace batch
}  // namespace sleefcu

// layout: Desc[kStaticItems], long long pre[kStaticItems + 1], tile counter
static __device__ __align__(256) unsigned char g_batch_scratch[kStaticBytes];

__global__ void __launch_bounds__(kStageItems) k_static_stage(const StageChunk c, Desc *d_desc, long long *d_pre,
                                                              unsigned long long *d_ctr) {
  int j = threadIdx.x;
  if (j < c.count) {
    d_desc[c.first + j] = c.desc[j];
    d_pre[c.first + j + 1] = c.pre[j];
  }
  if (c.first == 0 && j == 0) {
    d_pre[0] = 0;
    *d_ctr = 0;                          // the tile counter starts at 0 on every call
  }
}

extern "C" sleefcu_status sleefcu_batch_launch_static(const sleefcu_batch_item *items, size_t count,
                                                      sleefcu_stream s) {
  if (count > kStaticItems) {
    set_error("sleefcu_batch_launch_static: %zu items exceed the fixed scratch limit of %zu", count,
              kStaticItems);
    return SLEEFCU_EINVAL;
  }
  if (count && !items) { set_error("sleefcu_batch_launch_static: null item array"); return SLEEFCU_EINVAL; }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error("sleefcu_batch_launch_static: %s", cudaGetErrorString(e)); return SLEEFCU_ECUDA; }
  if (dev < 0 || dev >= kStaticMaxDevices) {
    set_error("sleefcu_batch_launch_static: device %d beyond the %d supported", dev, kStaticMaxDevices);
    return SLEEFCU_EUNSUPPORTED;
  }
  // every item is checked before anything is enqueued
  size_t nd = 0;
  long long ntiles = 0;
  for (size_t i = 0; i < count; i++) {
    const sleefcu_batch_item &it = items[i];
    int c = code_of(it);
    if (c < 0) {
      set_error("sleefcu_batch_launch_static: item %zu: unsupported (fn %u, dtype %u, ulp %u)", i, it.fn,
                it.dtype, it.ulp);
      return SLEEFCU_EUNSUPPORTED;
    }
    if (it.n == 0) continue;
    if (!it.x || !it.out || (needs_y(c) && !it.y) || (needs_out2(c) && !it.out2)) {
      set_error("sleefcu_batch_launch_static: item %zu: null pointer with n = %zu", i, it.n);
      return SLEEFCU_EINVAL;
    }
    if (sleefcu_status r = check_item("sleefcu_batch_launch_static", it, c)) return r;
    nd++;
    ntiles += (long long)((it.n + kStaticTile - 1) / kStaticTile);
  }
  if (ntiles == 0) return SLEEFCU_OK;
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_dev[dev]) {                             // first call on this device (device current)
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_batch_scratch);
      if (e != cudaSuccess || !p) {
        set_error("sleefcu_batch_launch_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return SLEEFCU_ECUDA;
      }
      g_static_dev[dev] = p;
    }
    addr = g_static_dev[dev];
  }
  unsigned char *base = (unsigned char *)addr;
  Desc *d_desc = (Desc *)base;
  long long *d_pre = (long long *)(base + kStaticDescBytes);
  unsigned long long *d_ctr = (unsigned long long *)(base + kStaticDescBytes + kStaticPreBytes);
  cudaStream_t st = (cudaStream_t)s;
  StageChunk chunk;
  chunk.first = 0;
  chunk.count = 0;
  long long pre = 0;
  size_t k = 0;
  for (size_t i = 0; i < count; i++) {
    const sleefcu_batch_item &it = items[i];
    if (it.n == 0) continue;
    pre += (long long)((it.n + kStaticTile - 1) / kStaticTile);
    chunk.desc[chunk.count] = Desc{it.x, it.y, it.out, it.out2, (long long)it.n, code_of(it), 0};
    chunk.pre[chunk.count] = pre;
    chunk.count++;
    k++;
    if (chunk.count == kStageItems || k == nd) {
      k_static_stage<<<1, kStageItems, 0, st>>>(chunk, d_desc, d_pre, d_ctr);
      if (sleefcu_status r = check_launch("sleefcu_batch_launch_static")) return r;
      chunk.first += chunk.count;
      chunk.count = 0;
    }
  }
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_batch, kStaticBlock, 0);
  if (per < 1) per = 1;
  long long g = (long long)sms * per * kStaticGridMult;
  if (g > ntiles) g = ntiles;
  if (g < 1) g = 1;
  k_batch<<<(int)g, kStaticBlock, 0, st>>>(d_desc, d_pre, (int)nd, ntiles, kStaticTile, kStaticVec, d_ctr);
  return check_launch("sleefcu_batch_launch_static");
}
