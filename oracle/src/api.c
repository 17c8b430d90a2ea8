/*
 * Registry and array forms of the oracle.
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * oracle_apply(name, x, y, out, out2, n, nthreads) evaluates the scalar
 * function `name` ("sin_u10_f64", ...) over n elements on nthreads POSIX
 * threads (static contiguous split).  Returns 0, or -1 for an unknown name.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>
#include "oracle.h"

enum { K_U64 = 1, K_B64 = 2, K_SC64 = 3, K_U32 = 11, K_B32 = 12, K_SC32 = 13, K_U16 = 21 };

typedef struct {
  const char *name;
  int kind;
  union {
    double (*u64)(double);
    double (*b64)(double, double);
    void (*sc64)(double, double *, double *);
    float (*u32)(float);
    float (*b32)(float, float);
    void (*sc32)(float, float *, float *);
    uint16_t (*u16)(uint16_t);
    void *any;
  } f;
} entry;

#define U64(n) { #n, K_U64, { .u64 = oracle_##n } }
#define B64(n) { #n, K_B64, { .b64 = oracle_##n } }
#define SC64(n) { #n, K_SC64, { .sc64 = oracle_##n } }
#define U32(n) { #n, K_U32, { .u32 = oracle_##n } }
#define B32(n) { #n, K_B32, { .b32 = oracle_##n } }
#define SC32(n) { #n, K_SC32, { .sc32 = oracle_##n } }
#define U16(n) { #n, K_U16, { .u16 = oracle_##n } }

static const entry REG[] = {
#include "registry.inc"
  { NULL, 0, { .any = NULL } }
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
