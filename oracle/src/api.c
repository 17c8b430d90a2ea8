/*
 * Registry and array forms of the oracle.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * oracle_apply(name, x, y, out, out2, n, nthreads) evaluates the scalar
 * function `name` ("sin_u10_f64", ...) over n elements on nthreads POSIX
 * threads (static contiguous split).  Returns 0, or -1 for an unknown name.
 * Group 0 is the function set of the vectorized method (registry.inc), group 1
 * the remaining C99 functions (registry_c99.inc), whose kinds include int32
 * operands and results (ilogb, ldexp, frexp).
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>
#include "oracle.h"

enum { K_U64 = 1, K_B64 = 2, K_SC64 = 3, K_UI64 = 4, K_BI64 = 5, K_SI64 = 6,
       K_U32 = 11, K_B32 = 12, K_SC32 = 13, K_UI32 = 14, K_BI32 = 15, K_SI32 = 16, K_U16 = 21 };

typedef struct {
  const char *name;
  int kind, grp;
  union {
    double (*u64)(double);
    double (*b64)(double, double);
    void (*sc64)(double, double *, double *);
    float (*u32)(float);
    float (*b32)(float, float);
    void (*sc32)(float, float *, float *);
    uint16_t (*u16)(uint16_t);
    int32_t (*ui64)(double);
    double (*bi64)(double, int32_t);
    double (*si64)(double, int32_t *);
    int32_t (*ui32)(float);
    float (*bi32)(float, int32_t);
    float (*si32)(float, int32_t *);
    void *any;
  } f;
} entry;

#define U64(n) { #n, K_U64, 0, { .u64 = oracle_##n } }
#define B64(n) { #n, K_B64, 0, { .b64 = oracle_##n } }
#define SC64(n) { #n, K_SC64, 0, { .sc64 = oracle_##n } }
#define U32(n) { #n, K_U32, 0, { .u32 = oracle_##n } }
#define B32(n) { #n, K_B32, 0, { .b32 = oracle_##n } }
#define SC32(n) { #n, K_SC32, 0, { .sc32 = oracle_##n } }
#define U16(n) { #n, K_U16, 0, { .u16 = oracle_##n } }

#define XU64(n) { #n, K_U64, 1, { .u64 = oracle_##n } }
#define XB64(n) { #n, K_B64, 1, { .b64 = oracle_##n } }
#define XSC64(n) { #n, K_SC64, 1, { .sc64 = oracle_##n } }
#define XUI64(n) { #n, K_UI64, 1, { .ui64 = oracle_##n } }
#define XBI64(n) { #n, K_BI64, 1, { .bi64 = oracle_##n } }
#define XSI64(n) { #n, K_SI64, 1, { .si64 = oracle_##n } }
#define XU32(n) { #n, K_U32, 1, { .u32 = oracle_##n } }
#define XB32(n) { #n, K_B32, 1, { .b32 = oracle_##n } }
#define XSC32(n) { #n, K_SC32, 1, { .sc32 = oracle_##n } }
#define XUI32(n) { #n, K_UI32, 1, { .ui32 = oracle_##n } }
#define XBI32(n) { #n, K_BI32, 1, { .bi32 = oracle_##n } }
#define XSI32(n) { #n, K_SI32, 1, { .si32 = oracle_##n } }

static const entry REG[] = {
#include "registry.inc"
#include "registry_c99.inc"
  { NULL, 0, 0, { .any = NULL } }
};

static const entry *find(const char *name) {
  for (const entry *e = REG; e->name; e++)
    if (!strcmp(e->name, name)) return e;
  return NULL;
}

int oracle_kind(const char *name) {
  const entry *e = find(name);
  return e ? e->kind : 0;
}

int oracle_count(void) { int n = 0; for (const entry *e = REG; e->name; e++) n++; return n; }
const char *oracle_name(int i) { return (i >= 0 && i < oracle_count()) ? REG[i].name : NULL; }
int oracle_group(int i) { return (i >= 0 && i < oracle_count()) ? REG[i].grp : -1; }

typedef struct {
  const entry *e; const void *x, *y; void *o, *o2; size_t lo, hi;
} job;

static void run(const job *j) {
  const entry *e = j->e;
  for (size_t i = j->lo; i < j->hi; i++) {
    switch (e->kind) {
      case K_U64: ((double *)j->o)[i] = e->f.u64(((const double *)j->x)[i]); break;
      case K_B64: ((double *)j->o)[i] = e->f.b64(((const double *)j->x)[i], ((const double *)j->y)[i]); break;
      case K_SC64: e->f.sc64(((const double *)j->x)[i], (double *)j->o + i, (double *)j->o2 + i); break;
      case K_U32: ((float *)j->o)[i] = e->f.u32(((const float *)j->x)[i]); break;
      case K_B32: ((float *)j->o)[i] = e->f.b32(((const float *)j->x)[i], ((const float *)j->y)[i]); break;
      case K_SC32: e->f.sc32(((const float *)j->x)[i], (float *)j->o + i, (float *)j->o2 + i); break;
      case K_U16: ((uint16_t *)j->o)[i] = e->f.u16(((const uint16_t *)j->x)[i]); break;
      case K_UI64: ((int32_t *)j->o)[i] = e->f.ui64(((const double *)j->x)[i]); break;
      case K_BI64: ((double *)j->o)[i] = e->f.bi64(((const double *)j->x)[i], ((const int32_t *)j->y)[i]); break;
      case K_SI64: ((double *)j->o)[i] = e->f.si64(((const double *)j->x)[i], (int32_t *)j->o2 + i); break;
      case K_UI32: ((int32_t *)j->o)[i] = e->f.ui32(((const float *)j->x)[i]); break;
      case K_BI32: ((float *)j->o)[i] = e->f.bi32(((const float *)j->x)[i], ((const int32_t *)j->y)[i]); break;
      case K_SI32: ((float *)j->o)[i] = e->f.si32(((const float *)j->x)[i], (int32_t *)j->o2 + i); break;
    }
  }
}

static void *thr(void *p) { run((const job *)p); return NULL; }

int oracle_apply(const char *name, const void *x, const void *y, void *out, void *out2,
                 size_t n, int nthreads) {
  const entry *e = find(name);
  if (!e) return -1;
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > n / 1024 + 1) nthreads = (int)(n / 1024 + 1);
  job *jobs = calloc((size_t)nthreads, sizeof(job));
  pthread_t *tid = calloc((size_t)nthreads, sizeof(pthread_t));
  size_t chunk = (n + (size_t)nthreads - 1) / (size_t)nthreads;
  for (int t = 0; t < nthreads; t++) {
    size_t lo = (size_t)t * chunk, hi = lo + chunk;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
    jobs[t] = (job){ e, x, y, out, out2, lo, hi };
  }
  for (int t = 1; t < nthreads; t++) pthread_create(&tid[t], NULL, thr, &jobs[t]);
  run(&jobs[0]);
  for (int t = 1; t < nthreads; t++) pthread_join(tid[t], NULL);
  free(jobs);
  free(tid);
  return 0;
}

/* Payne-Hanek reduction exported for the brute-force pin */
void oracle_ph_reduce(double x, int *q, double *hi, double *lo) {
  dd_t r = oracle_ph_reduce_dd(x, q);
  *hi = r.x;
  *lo = r.y;
}
