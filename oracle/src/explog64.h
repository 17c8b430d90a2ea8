/*
 * Internal cores of the FP64 exp/log oracle shared with the functions built
 * on them (exp2, exp10, expm1, log2, log10, log1p, the hyperbolics and their
 * inverses).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#ifndef ORACLE_EXPLOG64_H
#define ORACLE_EXPLOG64_H
#include "dd.h"

/* y 2^k in two multiplications by normal powers of two (one rounding) */
double oracle_scale2(double y, int k);
/* 2^k (1 + r + rl) with the 1-ULP exp polynomial; |r| <= ln2/2 (Section 5.6) */
double oracle_exp_tail_u10(double r, double rl, double k);
/* e^(Y - k ln2) - 1 as a DD and k = rint(Y.x / ln2), |Y.x| <= 746 */
dd_t oracle_expk_s(dd_t Y, double *k);
/* log m as a DD with a = m 2^e, m in [0.75, 1.5), for a DD a > 0 */
dd_t oracle_logm_u10(dd_t a, int *e);
/* the same in double for the 3.5-ULP forms */
double oracle_logm_u35(dd_t a, int *e);
double oracle_logm_u20(dd_t a, int *e);

/* log of a DD y > 0 with the 11-term DD polynomial of pow (about 2^-66) */
dd_t oracle_logk_dd(dd_t y);
/* e^Y for a DD Y with the DD exp of pow */
double oracle_exp_dd(dd_t Y);

#endif
