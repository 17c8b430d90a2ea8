// Device-side checks of the software binary64 arithmetic (softfp64.cuh)
// against the FP64 pipe of the GPU (__fma_rn, __dadd_rn, __dmul_rn, rint, trunc),
// bit for bit including the NaN pattern, and a throughput probe of the two.
// Test infrastructure, built by tests/test_softfp.py with nvcc.
#include <cuda_runtime.h>

#include "softfp_gen.h"

__global__ void k_check(uint64_t seed, long long per_thread, int mode_mask, unsigned long long *err,
                        unsigned long long *bad) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Rng r{seed + 0x632BE59BD9B4E019ull * (uint64_t)(tid + 1)};
  for (int mode = 0; mode < 8; mode++) {
    if (!(mode_mask & (1 << mode))) continue;
    for (long long i = 0; i < per_thread; i++) {
      uint64_t a, b, c;
      gen(r, mode, a, b, c);
      uint64_t got[5] = {S::fma(a, b, c), S::add(a, c), S::mul(a, b), S::rint(a), S::trunc(b)};
      uint64_t want[5] = {b_of(__fma_rn(d_of(a), d_of(b), d_of(c))), b_of(__dadd_rn(d_of(a), d_of(c))),
                          b_of(__dmul_rn(d_of(a), d_of(b))), b_of(rint(d_of(a))), b_of(trunc(d_of(b)))};
      for (int op = 0; op < 5; op++) {
        if (got[op] != want[op]) {
          // err[0]: any difference; err[1]: a difference that is not between two NaNs
          bool both_nan = is_nan(got[op]) && is_nan(want[op]);
          if (!both_nan) atomicAdd(err + 1, 1ull);
          if (atomicAdd(err, 1ull) == 0) {
            bad[0] = a; bad[1] = b; bad[2] = c; bad[3] = got[op]; bad[4] = want[op]; bad[5] = (uint64_t)op;
          }
        }
      }
    }
  }
}

// 8 independent chains of `iters` fused multiply-adds per thread, software
// or hardware; out gets one value per thread
// OP: 0 hardware fma, 1 software fma, 2 software add, 3 software mul,
// 4 hardware add, 5 hardware mul
template <int OP>
__global__ void k_tput(double *out, int iters, double a, double b) {
  double v[8];
#pragma unroll
  for (int j = 0; j < 8; j++) v[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (OP == 0) v[j] = __fma_rn(v[j], a, b);
      if (OP == 1) v[j] = d_of(S::fma(b_of(v[j]), b_of(a), b_of(b)));
      if (OP == 2) v[j] = d_of(S::add(b_of(v[j]), b_of(b)));
      if (OP == 3) v[j] = d_of(S::mul(b_of(v[j]), b_of(a)));
      if (OP == 4) v[j] = __dadd_rn(v[j], b);
      if (OP == 5) v[j] = __dmul_rn(v[j], a);
    }
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s += v[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" {
// blocks x 256 threads, per_thread triples per mode of mode_mask; d_err (2
// words: all differences, differences other than NaN payloads) and d_bad (6
// words: the first difference) are device memory, zeroed by the caller
int softfp_check_gpu(uint64_t seed, long long per_thread, int blocks, int mode_mask, unsigned long long *d_err,
                     unsigned long long *d_bad, void *stream) {
  if (blocks <= 0 || per_thread < 0 || !d_err || !d_bad) return -1;
  k_check<<<blocks, 256, 0, (cudaStream_t)stream>>>(seed, per_thread, mode_mask, d_err, d_bad);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int softfp_tput(int op, double *out, int blocks, int iters, void *stream) {
  if (blocks <= 0 || iters <= 0 || !out || op < 0 || op > 5) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  switch (op) {
    case 0: k_tput<0><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
    case 1: k_tput<1><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
    case 2: k_tput<2><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
    case 3: k_tput<3><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
    case 4: k_tput<4><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
    default: k_tput<5><<<blocks, 256, 0, s>>>(out, iters, 0.999999, 1e-7); break;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
}
