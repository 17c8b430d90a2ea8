/*
 * sleefcu — GB300 (sm_103a) elementwise C99 real math functions after the
 * method of Shibata & Petrogalli, "SLEEF: A Portable Vectorized Library of C
 * Standard Mathematical Functions", IEEE TPDS 31(6), 2020 (arXiv 2001.09258).
 *
 * C ABI.  Plain pointers and sizes; no C++ or framework types.
 *
 * Common conventions of every sleefcu_<fn>_<u10|u35>_<f64|f32> entry point:
 *  - x, y, out, out2 are DEVICE pointers owned by the caller; the library
 *    neither allocates nor frees them.  Host pointers are undefined behaviour
 *    in this library; the checked build (libsleefcu_checked.so, see the
 *    diagnostics section) rejects them with SLEEFCU_EINVAL.
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
 *    operation sequence (the bit-wise consistency of Section 4).
 *  - Accuracy: u10 entry points are within 1.0 ULP and u35 entry points
 *    within 3.5 ULP of the exact result (the two accuracy classes of Section
 *    2; lgamma near its negative-axis zeros has an absolute bound, see
 *    below).  Special values follow C99 Annex F; no
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
 * the vectorized Payne-Hanek reduction of Section 5.8 (table of the Payne-Hanek
 * table-generation figure) above that and for non-finite x; one sine
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

/* ---------------- exponential and logarithm, FP64 ----------------
 * exp (Section 5.6): x = k ln2 + r, |r| <= ln2/2, one polynomial for e^r
 * (13 terms u10, 11 terms u35), 2^k added to the exponent; exp(-inf) = +0,
 * exp(+inf) = +inf, overflow to +inf, underflow to 0 with subnormals rounded
 * once.
 * log (Section 5.5): subnormals rescaled by 2^64, e = floor(log2(4a/3)),
 * m = a 2^-e in [0.75, 1.5), log m = z + z^3 P(z^2) with z = 2(m-1)/(m+1);
 * log(+-0) = -inf, log(1) = +0, log(x < 0) = NaN, log(+inf) = +inf.
 * pow (Section 5.7): exp(y log|x|) with the logarithm and the product in
 * double-double; out[i] = pow(x[i], y[i]); every C99 Annex F special pair
 * (pow(x, +-0) = 1 even for NaN x, pow(+1, y) = 1, pow(x < 0, non-integer)
 * = NaN, zero and infinite bases and exponents).  The u35 entry point runs
 * the u10 algorithm. */
sleefcu_status sleefcu_exp_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_pow_u10_f64(const double *x, const double *y, double *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_pow_u35_f64(const double *x, const double *y, double *out, size_t n,
                                   sleefcu_stream stream);

/* ---------------- inverse trigonometric functions, FP64 ----------------
 * asin / acos (Section 5.3): |x| <= 0.5 directly, otherwise
 * asin x = pi/2 - 2 asin(sqrt((1-x)/2)), acos x = 2 asin(sqrt((1-x)/2))
 * (pi - that for x < -0.5); |x| > 1 gives NaN; asin(+-0) = +-0, acos(1) = +0.
 * atan (Section 5.4): 1/a for |a| >= 1 and pi/2 - atan(1/a);
 * atan(+-inf) = +-pi/2 (rounded), atan(+-0) = +-0.
 * atan2: out[i] = atan2(x[i], y[i]) with x the ordinate (C argument order);
 * all C99 Annex F special pairs (signed zeros select 0 or pi, infinities
 * select pi/4, 3pi/4, pi/2, 0 or pi). */
sleefcu_status sleefcu_asin_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asin_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acos_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acos_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u10_f64(const double *x, const double *y, double *out, size_t n,
                                     sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u35_f64(const double *x, const double *y, double *out, size_t n,
                                     sleefcu_stream stream);

/* ---------------- floating-point remainder, FP64 ----------------
 * fmod (Section 5.9, Algorithm 1 and the Appendix B listing): exact
 * x - trunc(x/y) y by long division with floating-point digits, the partial
 * remainder held exactly in double-double, one division in total; extended
 * to every pair of doubles (quotients up to 2^2098, at most 48 steps) by
 * dividing by power-of-two multiples of y while the quotient exceeds 2^1000.
 * out[i] = fmod(x[i], y[i]); sign of x; fmod(x, +-0) = NaN,
 * fmod(+-inf, y) = NaN, fmod(x, +-inf) = x for finite x.
 * remainder: x - n y with n the integer nearest x/y (ties to even), exact;
 * a zero result has the sign of x (IEEE 754 5.3.1); remainder(x, 0) and
 * remainder(inf, y) are NaN; remainder(x, +-inf) = x.
 * Results are exact, so u10 and u35 are the same operation. */
sleefcu_status sleefcu_fmod_u10_f64(const double *x, const double *y, double *out, size_t n,
                                    sleefcu_stream stream);
sleefcu_status sleefcu_fmod_u35_f64(const double *x, const double *y, double *out, size_t n,
                                    sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u10_f64(const double *x, const double *y, double *out, size_t n,
                                         sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u35_f64(const double *x, const double *y, double *out, size_t n,
                                         sleefcu_stream stream);

/* ---------------- functions built on the exp/log cores, FP64 ----------------
 * The paper lists these in the library without their steps; each is a fixed
 * IEEE sequence on the exp/log cores of Sections 5.5-5.7 with DD arithmetic
 * where the 1-ULP bound needs it (Section 3):
 * exp2 / exp10: k = rint(x) or rint(x log2 10), the reduced argument times
 *   ln2 or ln10 in DD, then the exp polynomial; overflow to +inf, underflow
 *   to 0 with subnormals rounded once; exp2(k) = 2^k and (u10) exp10(k) =
 *   10^k exactly where representable.
 * expm1: 2^k s + (2^k - 1) with s = e^r - 1 in DD; expm1(-0) = -0,
 *   expm1(-inf) = -1, expm1(x <= -40) = -1.
 * log2 / log10: the log core on the argument, times 1/ln2 or 1/ln10 in DD
 *   (u10) or rounded and one fma (u35); log2(2^k) = k, log10(10^k) = k;
 *   special values as log.  log1p: the log core on 1 + x formed exactly as
 *   a DD; log1p(-1) = -inf, log1p(x < -1) = NaN, log1p(+-0) = +-0.
 * cbrt: x = a 2^(3q), a in [1, 8); a division-free Newton step on a^(-1/3),
 *   then one Newton step on the root with the residual in DD (u10) or one
 *   fma (u35); cbrt(-x) = -cbrt(x), cbrt(+-0) = +-0, cbrt(+-inf) = +-inf.
 * sinh / cosh / tanh: from e^|x| - 1 (e^(2|x|) - 1 for tanh) in DD; sinh
 *   and cosh overflow only above 710.475; tanh(x) = +-1 for |x| > 20.
 * asinh / acosh / atanh: log of the DD argument |x| + sqrt(x^2+1),
 *   x + sqrt((x-1)(x+1)), (1+|x|)/(1-|x|); acosh(1) = +0, acosh(x < 1) = NaN,
 *   atanh(+-1) = +-inf, atanh(|x| > 1) = NaN.  Their u35 entry points run
 *   the u10 algorithm (no cheaper form keeps the cancellation exact).
 * Odd functions return -f(|x|) bit for bit; NaN results are the canonical
 * quiet NaN. */
sleefcu_status sleefcu_exp2_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp2_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log2_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log2_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log10_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log10_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);

/* erf / erfc, FP64: erf(x) = x (C0 + T (C1 + T (c2 + t P(t)))) for |x| < 1
 * (T = x^2 exact, outer levels in DD), 1 - erfc(|x|) up to 6, +-1 beyond;
 * erfc(x) = 1 -+ erf(|x|) for |x| < 1, else F(|x|) e^(-x^2) with
 * F = erfc e^(x^2) one polynomial per interval [1,2), [2,4), [4,8) and the
 * asymptotic factor G(1/x^2) / (sqrt(pi) x) from 8 on, e^(-x^2) in DD and
 * subnormal results rounded once; erfc(-x) = 2 - erfc(x); erfc(x > 27.3)
 * underflows to +0.  erf(+-0) = +-0, erf(+-inf) = +-1, erfc(-inf) = 2,
 * erfc(+inf) = +0.  The erfc u35 entry point runs the u10 algorithm. */
sleefcu_status sleefcu_erf_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);

/* tgamma / lgamma, FP64: log-gamma as a DD from Stirling's form (y >= 8,
 * with the DD logarithm of pow), polynomials about 2 and 1.5 (relative
 * accuracy across the zeros at 1 and 2), the shift y -> y + n with the
 * product in DD, and for y < 0 the reflection with sin(pi y) reduced
 * exactly; tgamma = exp of the DD log-gamma with the sign of sin(pi y).
 * tgamma(+-0) = +-inf, tgamma(negative integer or -inf) = NaN, overflow to
 * +inf above 171.62, underflow to +-0 below -190; lgamma(0 or a non-positive
 * integer or +-inf) = +inf, overflow to +inf above 2.556e305.  Near the
 * zeros of lgamma on the negative axis the error is bounded in absolute
 * terms (2^-51 max(1, |lgamma|)).  The u35 entry points run the u10
 * algorithm. */
sleefcu_status sleefcu_tgamma_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tgamma_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u10_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);

/* ---------------- masked FP64 entry points ----------------
 * The paper's whole-function opmask (Section 4): each FP64 entry point also
 * takes a mask of n bytes in device memory and evaluates only the elements
 * whose mask byte is non-zero; the other outputs are left as they are.  The
 * selected elements of each tile are gathered (and grouped by reduction
 * path) before they are evaluated, so the work scales with the number of
 * selected elements.  Results equal the unmasked entry point's bit for bit;
 * argument rules as for those (mask included). */
sleefcu_status sleefcu_sin_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_sin_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_cos_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_cos_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_tan_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_tan_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u10_f64_masked(const double *x, const uint8_t *mask, double *out_sin,
                                             double *out_cos, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u35_f64_masked(const double *x, const uint8_t *mask, double *out_sin,
                                             double *out_cos, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_exp_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_log_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_log_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_pow_u10_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                          size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_pow_u35_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                          size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asin_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_asin_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_acos_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_acos_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_atan_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_atan_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u10_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                            size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u35_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                            size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_fmod_u10_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                           size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_fmod_u35_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                           size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u10_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                                size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u35_f64_masked(const double *x, const double *y, const uint8_t *mask, double *out,
                                                size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp2_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_exp2_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_log2_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_log2_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_log10_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_log10_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                            sleefcu_stream stream);
sleefcu_status sleefcu_erf_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_erf_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                          sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                           sleefcu_stream stream);
sleefcu_status sleefcu_tgamma_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                             sleefcu_stream stream);
sleefcu_status sleefcu_tgamma_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                             sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u10_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                             sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u35_f64_masked(const double *x, const uint8_t *mask, double *out, size_t n,
                                             sleefcu_stream stream);

/* ---------------- FP32 family (float-float forms) ----------------
 * The same methods in binary32 arithmetic only, with float-float pairs where
 * the 1-ULP bound needs them (the paper describes the FP64 functions; "all
 * C99 real floating-point math functions" in both precisions, Section 1):
 * sin/cos (Cody-Waite for |x| < 2^20, the FF Payne-Hanek reduction with the
 * FP32 table above), exp, log, log1p (1 + x as an FF pair), tanh (via an FF
 * expm1) and erf (x P(x^2) below 1, 1 - exp(-x^2 + L(x)) above, +-1 from
 * 3.95).  Special values as for FP64; NaN results are 0x7FC00000. */
sleefcu_status sleefcu_sin_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sin_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cos_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cos_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);

/* The rest of the FP32 family: every FP64 function above also in binary32,
 * float-float where the 1-ULP bound needs it, no FP64 anywhere.  tan and
 * sincos reduce to quarter turns (Cody-Waite, the FF Payne-Hanek reduction
 * beyond 2^20) with one shared reduction for sincos; asin/acos/atan/atan2,
 * exp2/exp10/expm1, log2/log10, pow, cbrt, the hyperbolics and their
 * inverses, erfc, tgamma/lgamma follow the FP64 designs on the binary32
 * cores; fmod/remainder are exact (the long division with FF remainders, at
 * most 24 steps).  Special values as for FP64.  The u35 entry points of
 * expm1, sinh, cosh, asinh, acosh, atanh, pow, erfc, tgamma, lgamma, fmod and
 * remainder run the u10 algorithm. */
sleefcu_status sleefcu_tan_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tan_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u10_f32(const float *x, float *out_sin, float *out_cos, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_sincos_u35_f32(const float *x, float *out_sin, float *out_cos, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_asin_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asin_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acos_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acos_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u10_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_atan2_u35_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_pow_u10_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_pow_u35_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_fmod_u10_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_fmod_u35_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u10_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_remainder_u35_f32(const float *x, const float *y, float *out, size_t n,
                                   sleefcu_stream stream);
sleefcu_status sleefcu_exp2_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp2_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp10_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_expm1_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log2_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log2_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log10_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log10_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cbrt_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cosh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_asinh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_acosh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_atanh_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erfc_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tgamma_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tgamma_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u10_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_lgamma_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);

/* ---------------- bf16 / f16 activation forms ----------------
 * x and out hold n 16-bit values (bf16 or IEEE binary16, as the suffix says).
 * Each element is converted exactly to binary32, evaluated with the FP32
 * u10 / u35 entry point of the same name, and rounded to the 16-bit format
 * with round-to-nearest-even; NaN results are 0x7FC0 (bf16) / 0x7E00 (f16).
 * 16-byte-aligned arrays take the 8-elements-per-access path. */
sleefcu_status sleefcu_erf_u10_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u35_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u10_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u35_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u10_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u35_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u10_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u35_bf16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u10_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_erf_u35_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u10_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_tanh_u35_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u10_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_exp_u35_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u10_f16(const void *x, void *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_log1p_u35_f16(const void *x, void *out, size_t n, sleefcu_stream stream);

/* ---------------- batched mixed launch ----------------
 * Many arrays of uneven length, each with its own function, precision and
 * accuracy, evaluated by one persistent kernel (the batched form of the hot
 * path; every output equals the single-array entry point's, bit for bit).
 * fn: a sleefcu_fn; dtype: a sleefcu_dtype; ulp: 10 or 35.  x, y (binary
 * functions), out, out2 (sincos) are device pointers owned by the caller.
 * sleefcu_batch_create copies the descriptors to the device (it allocates
 * device memory and synchronizes; not capturable) and returns EUNSUPPORTED
 * for a combination the library does not have, EINVAL for a null pointer
 * with n > 0, ENOMEM when the descriptors do not fit.  Items with n == 0 are
 * ignored.  The caller keeps the arrays alive while the plan is launched.
 * tune_file_or_null: NULL keeps the default configuration (block 256, tile
 * 4096, grid multiplier 2, vector width 2); otherwise create ends with
 * sleefcu_batch_autotune(plan, tune_file_or_null, default stream) and waits
 * for it, with "" meaning "tune without a cache file" (the tuning runs write
 * the outputs).  Tuning is also its own call so that a plan can be re-tuned
 * (after sleefcu_batch_set_config, or on other data of the same shape).
 * sleefcu_batch_launch enqueues one memset and one kernel on the stream, no
 * allocation and no synchronization: it may be captured in a CUDA graph.
 * sleefcu_batch_launch_graph captures that pair once into a graph owned by
 * the plan and replays it on each call.  sleefcu_batch_autotune times the
 * candidate configurations (block size 128/256/512, 4/16/64 elements per
 * thread per tile, grid multiplier 1/2/4, vector width 1/2) on the plan's own
 * arrays (it overwrites the outputs) and keeps the fastest; with a cache file
 * (JSON lines keyed by device name and batch shape) a stored choice is reused
 * without timing.  Launches on one plan must not overlap (they share the
 * plan's tile counter). */
typedef enum {
  SLEEFCU_FN_SIN = 0, SLEEFCU_FN_COS, SLEEFCU_FN_TAN, SLEEFCU_FN_SINCOS, SLEEFCU_FN_ASIN,
  SLEEFCU_FN_ACOS, SLEEFCU_FN_ATAN, SLEEFCU_FN_ATAN2, SLEEFCU_FN_EXP, SLEEFCU_FN_LOG, SLEEFCU_FN_POW,
  SLEEFCU_FN_FMOD, SLEEFCU_FN_REMAINDER, SLEEFCU_FN_LOG1P, SLEEFCU_FN_TANH, SLEEFCU_FN_ERF,
  SLEEFCU_FN_EXP2, SLEEFCU_FN_EXP10, SLEEFCU_FN_EXPM1, SLEEFCU_FN_LOG2, SLEEFCU_FN_LOG10,
  SLEEFCU_FN_CBRT, SLEEFCU_FN_SINH, SLEEFCU_FN_COSH, SLEEFCU_FN_ASINH, SLEEFCU_FN_ACOSH,
  SLEEFCU_FN_ATANH, SLEEFCU_FN_ERFC, SLEEFCU_FN_TGAMMA, SLEEFCU_FN_LGAMMA,
  SLEEFCU_FN_COUNT
} sleefcu_fn;
typedef enum { SLEEFCU_F64 = 0, SLEEFCU_F32 = 1, SLEEFCU_BF16 = 2, SLEEFCU_F16 = 3 } sleefcu_dtype;
typedef struct {
  uint16_t fn;
  uint8_t dtype;
  uint8_t ulp;
  uint32_t reserved;
  const void *x;
  const void *y;
  void *out;
  void *out2;
  size_t n;
} sleefcu_batch_item;
typedef struct sleefcu_batch sleefcu_batch;

sleefcu_status sleefcu_batch_create(const sleefcu_batch_item *items, size_t count, const char *tune_file_or_null,
                                    sleefcu_batch **plan);
sleefcu_status sleefcu_batch_launch(sleefcu_batch *plan, sleefcu_stream stream);
sleefcu_status sleefcu_batch_launch_graph(sleefcu_batch *plan, sleefcu_stream stream);
sleefcu_status sleefcu_batch_autotune(sleefcu_batch *plan, const char *cache_file_or_null, sleefcu_stream stream);
sleefcu_status sleefcu_batch_set_config(sleefcu_batch *plan, int block, int tile, int grid_mult, int vec);
sleefcu_status sleefcu_batch_get_config(const sleefcu_batch *plan, int *block, int *tile, int *grid_mult,
                                        int *vec);
void sleefcu_batch_destroy(sleefcu_batch *plan);

/* Batched launch without allocation (this library's addition; the paper has
 * no counterpart).  The same evaluation as a plan's sleefcu_batch_launch,
 * bit for bit, for callers that may not allocate device memory when they
 * launch: an application whose caching allocator owns the device heap (a
 * cudaMalloc of its own would fragment it or fail), or a latency-critical
 * path that cannot take cudaMalloc/cudaFree and the synchronization they
 * imply.  The descriptors, tile prefix sums and tile counter live in one
 * fixed device array of about 230 KB inside the library instead of
 * cudaMalloc'd plan buffers; every GPU that loads the library holds it
 * until the process exits.  items: host array of count descriptors (the
 * same rules as sleefcu_batch_create; items with n == 0 are skipped).
 * count > 4096 returns SLEEFCU_EINVAL with a message; an unsupported
 * combination SLEEFCU_EUNSUPPORTED; every item is checked before anything
 * is enqueued.  The call enqueues ceil(items with n > 0 / 512) small staging
 * kernels, which carry the descriptors as kernel arguments and also zero
 * the tile counter, then the batched kernel, in that order on `stream`, and
 * returns without waiting for the stream (there is no copy from host
 * memory); the configuration is the default one (block 256, tile 4096).
 * The first call on each device looks up the array's address with that
 * device current; make that first call before any stream capture.  One
 * array serves all callers on a device and keeps the last call's contents:
 * calls whose work can overlap on the GPU (other streams, other host
 * threads) race on it and corrupt each other's descriptors; serialize them
 * on one stream or synchronize in between.  Nothing is allocated, by this
 * call or the first one. */
sleefcu_status sleefcu_batch_launch_static(const sleefcu_batch_item *items, size_t count,
                                           sleefcu_stream stream);

/* ---------------- evaluation from host memory ----------------
 * The end-to-end form of every entry point: item describes one array exactly
 * as for the batched launch, but x, y, out, out2 are HOST pointers.  The
 * library streams the arrays through device buffers it owns in chunks of
 * `chunk` elements (0: 4,194,304), keeping up to six chunks in flight:
 * copies in, the entry point's kernels and copies out run concurrently on
 * three library streams.  Results equal the device
 * entry point's bit for bit.  The call is synchronous: it returns when out
 * (and out2) hold every result.  Host arrays should be page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to overlap; pageable
 * memory works at lower speed.  The staging buffers (6 x 4 x chunk x element
 * size bytes of device memory) and streams are created on the first call
 * per device and kept; ENOMEM if they cannot be allocated.  Calls from
 * several host threads on one device are serialized. */
sleefcu_status sleefcu_eval_host(const sleefcu_batch_item *item, size_t chunk);

/* The same for `count` host arrays in one call: the chunks of all items go
 * through one pipeline in item order, so the copy in of an item's first
 * chunk overlaps the kernels of the previous item's last ones (a loop of
 * sleefcu_eval_host calls drains the pipeline at every item).  Every item
 * is checked before any work starts: EINVAL for a null items with count > 0
 * or a null pointer with n > 0, EUNSUPPORTED for an unknown (fn, dtype, ulp);
 * count == 0 returns OK.  Synchronous like sleefcu_eval_host; same staging
 * buffers. */
sleefcu_status sleefcu_eval_host_many(const sleefcu_batch_item *items, size_t count, size_t chunk);

/* ---------------- diagnostics (not part of the method) ----------------
 * The checked build (libsleefcu_checked.so, compiled with -DSLEEFCU_CHECKED
 * from the same sources) has every entry point of this header with the same
 * results, plus checks that cost time: before any launch, each device
 * pointer argument is looked up (cudaPointerGetAttributes and the
 * allocation's address range) and the call returns SLEEFCU_EINVAL, with a
 * message, for host memory, memory of another device, or an array whose n
 * elements run past the end of its allocation (sleefcu_eval_host and
 * sleefcu_eval_host_many, which take host arrays, are not checked); and the
 * kernels count table indices that had to be clamped for a finite argument
 * (the Payne-Hanek table gathers; a non-zero count means a lane reached the
 * gather on a path it should not take), without trapping.
 * sleefcu_is_checked: 1 in the checked build, 0 in the normal one.
 * sleefcu_checked_error_count: the count since the last reset, summed over
 * the library's kernels on the current device (synchronous: it reads device
 * memory); reset != 0 zeroes it.  EINVAL for a null count; in the normal
 * build it returns SLEEFCU_EUNSUPPORTED. */
int sleefcu_is_checked(void);
sleefcu_status sleefcu_checked_error_count(unsigned long long *count, int reset);


/* Long-division step count of the remainder kernels (Section 5.9): out[i] =
 * the number of steps the fmod kernel takes for |x[i]| mod |y[i]| (0 where
 * x[i] is not finite or y[i] is 0 or not finite), as a double.  For
 * remainder(x, y) pass 2|y|.  Used for the algorithmic operation count of
 * the roofline; the same argument rules as the math entry points. */
sleefcu_status sleefcu_fmod_steps_f64(const double *x, const double *y, double *out, size_t n,
                                      sleefcu_stream stream);

/* ---------------- the remaining C99 real functions ----------------
 * The library's claim to the whole C99 real set (Section 1): the functions
 * below complete it beside the families above.  Conventions as at the top of
 * this file (device pointers owned by the caller, any alignment, n == 0 is a
 * no-op, null with n > 0 is SLEEFCU_EINVAL, asynchronous on stream), with
 * int32_t arrays where C99 has an int.
 *
 * Exact functions (no accuracy tag; the result is the exact value, or the
 * correctly rounded one where C99 rounds): fabs, copysign, fmax, fmin, fdim,
 * trunc, floor, ceil, round (ties away from zero), rint (ties to even),
 * nextafter, logb, ilogb, ldexp, frexp, modf.  Every NaN result is the
 * canonical quiet NaN (fabs and copysign included).
 * Choices C99 leaves to the implementation:
 *   fmax(+0, -0) = fmax(-0, +0) = +0 and fmin(+0, -0) = fmin(-0, +0) = -0;
 *   fmax / fmin with one NaN operand return the other operand;
 *   ilogb(+-0) = SLEEFCU_FP_ILOGB0, ilogb(NaN) = SLEEFCU_FP_ILOGBNAN,
 *   ilogb(+-inf) = INT32_MAX; logb(+-0) = -inf, logb(+-inf) = +inf;
 *   frexp(+-0, +-inf, NaN) returns x (NaN canonical) and stores 0;
 *   modf(+-inf) = (+-0, +-inf); ldexp rounds once, overflow gives +-inf.
 *
 * sqrt_u05 / sqrt_u35: the IEEE square root (correctly rounded; the u35 entry
 * point runs the same sequence).  sqrt(-0) = -0, sqrt(x < 0) = NaN.
 * hypot_u05 (<= 0.5 + 2^-20 ULP for normal results, <= 1 ULP for subnormal
 * ones) and hypot_u35 (<= 1 ULP): the larger magnitude's exponent is taken out
 * exactly, the sum of squares and its square root in double-double
 * (float-float) arithmetic (u05) or one fma and a square root (u35).
 * hypot(+-inf, y) = +inf even for a NaN y; hypot(x, +-0) = |x|.
 * sinpi_u05 / cospi_u05 (<= 0.501 ULP for normal results, <= 1 ULP for
 * subnormal ones) and the u35 forms (<= 2 ULP): sin(pi x) and cos(pi x) from
 * the exact reduction x = q/2 + s, |s| <= 1/4, and one polynomial shape whose
 * coefficients the quadrant selects.  sinpi(+-n) = +-0 for integers n,
 * cospi(n + 1/2) = +0, cospi(+-0) = 1, +-inf and NaN give NaN. */
#define SLEEFCU_FP_ILOGB0 INT32_MIN
#define SLEEFCU_FP_ILOGBNAN INT32_MAX
sleefcu_status sleefcu_fabs_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_trunc_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_floor_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_ceil_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_round_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_rint_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_logb_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sqrt_u05_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sqrt_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinpi_u05_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinpi_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cospi_u05_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cospi_u35_f64(const double *x, double *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_copysign_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fmax_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fmin_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fdim_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_nextafter_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_hypot_u05_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_hypot_u35_f64(const double *x, const double *y, double *out, size_t n,
                               sleefcu_stream stream);
/* modf: frac[i] = the fractional part (sign of x[i]), ipart[i] = the integral part */
sleefcu_status sleefcu_modf_f64(const double *x, double *frac, double *ipart, size_t n, sleefcu_stream stream);
/* ilogb: out[i] = the unbiased exponent of x[i] */
sleefcu_status sleefcu_ilogb_f64(const double *x, int32_t *out, size_t n, sleefcu_stream stream);
/* ldexp: out[i] = x[i] 2^e[i], rounded once */
sleefcu_status sleefcu_ldexp_f64(const double *x, const int32_t *e, double *out, size_t n,
                               sleefcu_stream stream);
/* frexp: x[i] = m[i] 2^e[i] with |m[i]| in [1/2, 1) */
sleefcu_status sleefcu_frexp_f64(const double *x, double *m, int32_t *e, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_fabs_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_trunc_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_floor_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_ceil_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_round_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_rint_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_logb_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sqrt_u05_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sqrt_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinpi_u05_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_sinpi_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cospi_u05_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_cospi_u35_f32(const float *x, float *out, size_t n, sleefcu_stream stream);
sleefcu_status sleefcu_copysign_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fmax_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fmin_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_fdim_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_nextafter_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_hypot_u05_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
sleefcu_status sleefcu_hypot_u35_f32(const float *x, const float *y, float *out, size_t n,
                               sleefcu_stream stream);
/* modf: frac[i] = the fractional part (sign of x[i]), ipart[i] = the integral part */
sleefcu_status sleefcu_modf_f32(const float *x, float *frac, float *ipart, size_t n, sleefcu_stream stream);
/* ilogb: out[i] = the unbiased exponent of x[i] */
sleefcu_status sleefcu_ilogb_f32(const float *x, int32_t *out, size_t n, sleefcu_stream stream);
/* ldexp: out[i] = x[i] 2^e[i], rounded once */
sleefcu_status sleefcu_ldexp_f32(const float *x, const int32_t *e, float *out, size_t n,
                               sleefcu_stream stream);
/* frexp: x[i] = m[i] 2^e[i] with |m[i]| in [1/2, 1) */
sleefcu_status sleefcu_frexp_f32(const float *x, float *m, int32_t *e, size_t n, sleefcu_stream stream);

#ifdef __cplusplus
}
#endif
#endif
