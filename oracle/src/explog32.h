/*
 * Internal FP32 (float-float) cores of the oracle shared by the FP32
 * functions built on exp and log.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#ifndef ORACLE_EXPLOG32_H
#define ORACLE_EXPLOG32_H
#include "dd.h"

float oracle_scale2f(float y, int k);
float oracle_expf_tail_u10(float r, float rl, float k);
ff_t oracle_expf_parts(ff_t a, float *k);
ff_t oracle_expm1f_s(float a, float *k);
ff_t oracle_logmf_u10(ff_t a, int *e);
float oracle_logmf_u20(ff_t a, int *e);
ff_t oracle_logf_ff(ff_t a);
ff_t oracle_logkf(ff_t a);
ff_t oracle_erfcf_L(float x);
ff_t oracle_erff_a(float a);
ff_t oracle_erfcf_a(float a);

#endif
