/*
 * Scalar C oracle of the vectorized libm method (Shibata & Petrogalli,
 * "SLEEF", IEEE TPDS 2020).  Test infrastructure: only tests/, the smoke
 * check and the CPU-baseline leg of the benchmark may use anything under
 * oracle/.  Compiled with -ffp-contract=off -fno-fast-math; fma() only where
 * written; round-to-nearest only (Section 5.10).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>
#include "common.h"

double oracle_sin_u10_f64(double);
double oracle_sin_u35_f64(double);
double oracle_cos_u10_f64(double);
double oracle_cos_u35_f64(double);
double oracle_tan_u10_f64(double);
double oracle_tan_u35_f64(double);
void oracle_sincos_u10_f64(double, double *, double *);
void oracle_sincos_u35_f64(double, double *, double *);

double oracle_exp_u10_f64(double);
double oracle_exp_u35_f64(double);
double oracle_log_u10_f64(double);
double oracle_log_u35_f64(double);
double oracle_exp2_u10_f64(double);
double oracle_exp2_u35_f64(double);
double oracle_exp10_u10_f64(double);
double oracle_exp10_u35_f64(double);
double oracle_expm1_u10_f64(double);
double oracle_expm1_u35_f64(double);
double oracle_log2_u10_f64(double);
double oracle_log2_u35_f64(double);
double oracle_log10_u10_f64(double);
double oracle_log10_u35_f64(double);
double oracle_log1p_u10_f64(double);
double oracle_log1p_u35_f64(double);
double oracle_cbrt_u10_f64(double);
double oracle_cbrt_u35_f64(double);
double oracle_sinh_u10_f64(double);
double oracle_sinh_u35_f64(double);
double oracle_cosh_u10_f64(double);
double oracle_cosh_u35_f64(double);
double oracle_tanh_u10_f64(double);
double oracle_tanh_u35_f64(double);
double oracle_asinh_u10_f64(double);
double oracle_asinh_u35_f64(double);
double oracle_acosh_u10_f64(double);
double oracle_acosh_u35_f64(double);
double oracle_atanh_u10_f64(double);
double oracle_atanh_u35_f64(double);
double oracle_erf_u10_f64(double);
double oracle_erf_u35_f64(double);
double oracle_erfc_u10_f64(double);
double oracle_erfc_u35_f64(double);
double oracle_tgamma_u10_f64(double);
double oracle_tgamma_u35_f64(double);
double oracle_lgamma_u10_f64(double);
double oracle_lgamma_u35_f64(double);
double oracle_pow_u10_f64(double, double);
double oracle_pow_u35_f64(double, double);
double oracle_asin_u10_f64(double);
double oracle_asin_u35_f64(double);
double oracle_acos_u10_f64(double);
double oracle_acos_u35_f64(double);
double oracle_atan_u10_f64(double);
double oracle_atan_u35_f64(double);
double oracle_atan2_u10_f64(double, double);
double oracle_atan2_u35_f64(double, double);

double oracle_fmod_u10_f64(double, double);
double oracle_fmod_u35_f64(double, double);
double oracle_remainder_u10_f64(double, double);
double oracle_remainder_u35_f64(double, double);
int oracle_fmod_iters(double, double);
double oracle_fmod_recip(double);
int oracle_fmod_trace(double, double, double *, double *, int);

float oracle_sin_u10_f32(float);
float oracle_sin_u35_f32(float);
float oracle_cos_u10_f32(float);
float oracle_cos_u35_f32(float);
float oracle_exp2_u10_f32(float);
float oracle_exp2_u35_f32(float);
float oracle_exp10_u10_f32(float);
float oracle_exp10_u35_f32(float);
float oracle_expm1_u10_f32(float);
float oracle_expm1_u35_f32(float);
float oracle_log2_u10_f32(float);
float oracle_log2_u35_f32(float);
float oracle_log10_u10_f32(float);
float oracle_log10_u35_f32(float);
float oracle_sinh_u10_f32(float);
float oracle_sinh_u35_f32(float);
float oracle_cosh_u10_f32(float);
float oracle_cosh_u35_f32(float);
float oracle_asinh_u10_f32(float);
float oracle_asinh_u35_f32(float);
float oracle_acosh_u10_f32(float);
float oracle_acosh_u35_f32(float);
float oracle_atanh_u10_f32(float);
float oracle_atanh_u35_f32(float);
float oracle_cbrt_u10_f32(float);
float oracle_cbrt_u35_f32(float);
float oracle_erfc_u10_f32(float);
float oracle_erfc_u35_f32(float);
float oracle_pow_u10_f32(float, float);
float oracle_pow_u35_f32(float, float);
float oracle_tan_u10_f32(float);
float oracle_tan_u35_f32(float);
float oracle_asin_u10_f32(float);
float oracle_asin_u35_f32(float);
float oracle_acos_u10_f32(float);
float oracle_acos_u35_f32(float);
float oracle_atan_u10_f32(float);
float oracle_atan_u35_f32(float);
float oracle_tgamma_u10_f32(float);
float oracle_tgamma_u35_f32(float);
float oracle_lgamma_u10_f32(float);
float oracle_lgamma_u35_f32(float);
float oracle_atan2_u10_f32(float, float);
float oracle_atan2_u35_f32(float, float);
float oracle_fmod_u10_f32(float, float);
float oracle_fmod_u35_f32(float, float);
float oracle_remainder_u10_f32(float, float);
float oracle_remainder_u35_f32(float, float);
void oracle_sincos_u10_f32(float, float *, float *);
void oracle_sincos_u35_f32(float, float *, float *);
float oracle_exp_u10_f32(float);
float oracle_exp_u35_f32(float);
float oracle_log_u10_f32(float);
float oracle_log_u35_f32(float);
float oracle_log1p_u10_f32(float);
float oracle_log1p_u35_f32(float);
float oracle_tanh_u10_f32(float);
float oracle_tanh_u35_f32(float);
float oracle_erf_u10_f32(float);
float oracle_erf_u35_f32(float);
void oracle_ph_reduce_f32(float, int *, float *, float *);

uint16_t oracle_erf_u10_bf16(uint16_t);
uint16_t oracle_erf_u10_f16(uint16_t);
uint16_t oracle_erf_u35_bf16(uint16_t);
uint16_t oracle_erf_u35_f16(uint16_t);
uint16_t oracle_tanh_u10_bf16(uint16_t);
uint16_t oracle_tanh_u10_f16(uint16_t);
uint16_t oracle_tanh_u35_bf16(uint16_t);
uint16_t oracle_tanh_u35_f16(uint16_t);
uint16_t oracle_exp_u10_bf16(uint16_t);
uint16_t oracle_exp_u10_f16(uint16_t);
uint16_t oracle_exp_u35_bf16(uint16_t);
uint16_t oracle_exp_u35_f16(uint16_t);
uint16_t oracle_log1p_u10_bf16(uint16_t);
uint16_t oracle_log1p_u10_f16(uint16_t);
uint16_t oracle_log1p_u35_bf16(uint16_t);
uint16_t oracle_log1p_u35_f16(uint16_t);
float oracle_bf16_to_f32(uint16_t);
uint16_t oracle_f32_to_bf16(float);
float oracle_f16_to_f32(uint16_t);
uint16_t oracle_f32_to_f16(float);

/* the remaining C99 set (c99ext.c) */
double oracle_fabs_f64(double);
double oracle_trunc_f64(double);
double oracle_floor_f64(double);
double oracle_ceil_f64(double);
double oracle_round_f64(double);
double oracle_rint_f64(double);
double oracle_logb_f64(double);
double oracle_sqrt_u05_f64(double);
double oracle_sqrt_u35_f64(double);
double oracle_sinpi_u05_f64(double);
double oracle_sinpi_u35_f64(double);
double oracle_cospi_u05_f64(double);
double oracle_cospi_u35_f64(double);
double oracle_copysign_f64(double, double);
double oracle_fmax_f64(double, double);
double oracle_fmin_f64(double, double);
double oracle_fdim_f64(double, double);
double oracle_nextafter_f64(double, double);
double oracle_hypot_u05_f64(double, double);
double oracle_hypot_u35_f64(double, double);
void oracle_modf_f64(double, double *, double *);
int32_t oracle_ilogb_f64(double);
double oracle_ldexp_f64(double, int32_t);
double oracle_frexp_f64(double, int32_t *);
float oracle_fabs_f32(float);
float oracle_trunc_f32(float);
float oracle_floor_f32(float);
float oracle_ceil_f32(float);
float oracle_round_f32(float);
float oracle_rint_f32(float);
float oracle_logb_f32(float);
float oracle_sqrt_u05_f32(float);
float oracle_sqrt_u35_f32(float);
float oracle_sinpi_u05_f32(float);
float oracle_sinpi_u35_f32(float);
float oracle_cospi_u05_f32(float);
float oracle_cospi_u35_f32(float);
float oracle_copysign_f32(float, float);
float oracle_fmax_f32(float, float);
float oracle_fmin_f32(float, float);
float oracle_fdim_f32(float, float);
float oracle_nextafter_f32(float, float);
float oracle_hypot_u05_f32(float, float);
float oracle_hypot_u35_f32(float, float);
void oracle_modf_f32(float, float *, float *);
int32_t oracle_ilogb_f32(float);
float oracle_ldexp_f32(float, int32_t);
float oracle_frexp_f32(float, int32_t *);

int oracle_apply(const char *name, const void *x, const void *y, void *out, void *out2,
                 size_t n, int nthreads);
#endif
