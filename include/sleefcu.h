/*
 * sleefcu — GB300 (sm_103a) elementwise C99 real math functions after the
 * method of Shibata & Petrogalli, "SLEEF: A Portable Vectorized Library of C
 * Standard Mathematical Functions", IEEE TPDS 31(6), 2020 (arXiv 2001.09258).
 *
 * C ABI.  Plain pointers and sizes; no C++ or framework types.
 *
 * Common conventions of every sleefcu_<fn>_<u10|u35>_<f64|f32> entry point:
 *  - x, y, out, out2 are DEVICE pointers owned by the caller; the library
 *    neither allocates nor frees them.  Host pointers are undefined behaviour.
 *  - Layout: contiguous 1-D arrays of n elements.  Any alignment is accepted
 *    (16-byte-aligned arrays take the vectorized path).  out may equal x
 *    (in place); any other overlap between inputs and outputs is undefined.
 *  - n == 0 returns SLEEFCU_OK and may pass null pointers.  A null pointer
 *    with n > 0 returns SLEEFCU_EINVAL.
 *  - stream is a cudaStream_t (NULL = the legacy default stream).  The call
 *    is asynchronous on it and performs no allocation and no synchronization.
 *    A launch failure returns SLEEFCU_ECUDA; sleefcu_last_error() then holds
 *    the CUDA error text (thread-local).
 *  - Results are deterministic: the same bits for any launch configuration,
 *    and the same bits as the scalar reference implementation of the same
 *    operation sequence (Section 4, "Making Results Bit-wise Consistent").
 *  - Accuracy: u10 entry points are within 1.0 ULP and u35 entry points
 *    within 3.5 ULP of the exact result (Section 2: "1-ULP accuracy version
 *    and 3.5-ULP accuracy version").  Special values follow C99 Annex F; no
 *    errno, no floating-point flags, round-to-nearest only (Section 5.10).
 *    Every NaN result is the canonical quiet NaN (0x7FF8000000000000 /
 *    0x7FC00000).
 *  - Binary functions take C argument order: out[i] = f(x[i], y[i]).
 */
#ifndef SLEEFCU_H
#define SLEEFCU_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SLEEFCU_OK = 0,
  SLEEFCU_EINVAL = -1,        /* null pointer with n > 0, bad argument */
  SLEEFCU_ECUDA = -2,         /* CUDA launch or runtime error */
  SLEEFCU_EUNSUPPORTED = -3,  /* no sm_103a device or unknown function */
  SLEEFCU_ENOMEM = -4
} sleefcu_status;

typedef void *sleefcu_stream;   /* a cudaStream_t */

/* Thread-local text of the last error returned on this thread ("" if none). */
const char *sleefcu_last_error(void);
/* Library version string. */
const char *sleefcu_version(void);

/* ---------------- trigonometric functions, FP64 ----------------
 * Section 5.1 (sin, cos): Cody-Waite reduction for |x| < 15 and |x| < 1e14,
 * the vectorized Payne-Hanek reduction of Section 5.8 (table of Fig.
 * "Payne-Hanek table generation") above that and for non-finite x; one sine
 * polynomial on [-pi/2, pi/2]; the sign is set in the reconstruction.
 * Section 5.2 and Appendix A (tan): the same reductions to quarter turns,
 * half-angle reduction, tan polynomial, double-angle reconstruction.
 * sincos writes sin(x[i]) to out_sin[i] and cos(x[i]) to out_cos[i] from one
 * shared quarter-turn reduction.
 * sin(+-0) = +-0, tan(+-0) = +-0, cos(+-0) = 1; +-inf and NaN give NaN. */
sleefcu_status sleefcu_sin_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sin_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cos_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cos_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tan_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tan_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u10_f64(const double *x, double *out_sin, double *out_cos, size_t n,
                                      sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u35_f64(const double *x, double *out_sin, double *out_cos, size_t n,
                                      sleefcu_stream stream);

/* ---------------- diagnostics (not part of the method) ----------------
 * Pipe-throughput probes for the roofline denominators: blocks x 256 threads
 * each run 8 independent chains of `iters` fused multiply-adds in FP64
 * (probe_dfma) or FP32 (probe_ffma), i.e. blocks*256*iters*8 FMAs, and write
 * one value per thread to out (blocks*256 elements, device memory owned by
 * the caller).  EINVAL for a null out or non-positive blocks / iters. */
sleefcu_status sleefcu_probe_dfma(double *out, int blocks, int iters, sleefcu_stream stream);
sleefcu_status sleefcu_probe_ffma(float *out, int blocks, int iters, sleefcu_stream stream);

#ifdef __cplusplus
}
#endif
#endif
