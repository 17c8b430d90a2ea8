// Pipe-throughput probes for the roofline denominators of bench.py (not part
// of the library): blocks x 256 threads each run 8 independent chains of
// `iters` fused multiply-adds in FP64 (probe_dfma) or FP32 (probe_ffma),
// blocks*256*iters*8 FMAs in all, and write one value per thread to `out`
// (blocks*256 elements of device memory owned by the caller).  Returns 0, -1
// for a null out or non-positive blocks / iters, -2 for a launch error.
#include <cuda_runtime.h>

namespace {
constexpr int kBlock = 256;

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
}  // namespace

extern "C" int probe_dfma(double *out, int blocks, int iters, void *stream) {
  if (!out || blocks <= 0 || iters <= 0) return -1;
  k_probe_dfma<<<blocks, kBlock, 0, (cudaStream_t)stream>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int probe_ffma(float *out, int blocks, int iters, void *stream) {
  if (!out || blocks <= 0 || iters <= 0) return -1;
  k_probe_ffma<<<blocks, kBlock, 0, (cudaStream_t)stream>>>(out, iters, 0.999999f, 1e-7f);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
