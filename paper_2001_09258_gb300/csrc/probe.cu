// Diagnostic kernels (not part of the method): throughput probes used to
// measure the FP64 and FP32 pipe peaks of the device that the roofline of
// the FP64 / FP32 families is quoted against.
#include "sleefcu_common.cuh"

namespace sleefcu {
// each thread runs 8 independent chains of `iters` fused multiply-adds
__global__ void __launch_bounds__(kBlock) k_probe_dfma(double *out, int iters, double a, double b) {
  double v[8];
#pragma unroll
  for (int j = 0; j < 8; j++) v[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = __fma_rn(v[j], a, b);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s += v[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void __launch_bounds__(kBlock) k_probe_ffma(float *out, int iters, float a, float b) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; j++) v[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = __fmaf_rn(v[j], a, b);
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s += v[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace sleefcu

// out: blocks * 256 elements of scratch owned by the caller; performs
// blocks * 256 * iters * 8 fused multiply-adds.
extern "C" sleefcu_status sleefcu_probe_dfma(double *out, int blocks, int iters, sleefcu_stream s) {
  if (!out || blocks <= 0 || iters <= 0) { sleefcu::set_error("sleefcu_probe_dfma: bad argument"); return SLEEFCU_EINVAL; }
  sleefcu::k_probe_dfma<<<blocks, sleefcu::kBlock, 0, (cudaStream_t)s>>>(out, iters, 0.999999, 1e-7);
  return sleefcu::check_launch("sleefcu_probe_dfma");
}
extern "C" sleefcu_status sleefcu_probe_ffma(float *out, int blocks, int iters, sleefcu_stream s) {
  if (!out || blocks <= 0 || iters <= 0) { sleefcu::set_error("sleefcu_probe_ffma: bad argument"); return SLEEFCU_EINVAL; }
  sleefcu::k_probe_ffma<<<blocks, sleefcu::kBlock, 0, (cudaStream_t)s>>>(out, iters, 0.999999f, 1e-7f);
  return sleefcu::check_launch("sleefcu_probe_ffma");
}
