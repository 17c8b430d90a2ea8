/*
 * Exhaustive accuracy check of the oracle's binary32 functions (test
 * infrastructure): every one of the 2^32 binary32 inputs x, the binary32
 * result y = f32(x) against the binary64 oracle's r = f64(x) (x widened
 * exactly), in units of the binary32 ulp of r:
 *   ulp(r) = 2^(max(floor(log2 |r|), -126) - 23)     (the ULP definition, reading R5)
 * The binary64 reference is itself within 1 binary64 ulp of the exact value,
 * which is 2^-29 binary32 ulp: the bound the test asserts carries that slack.
 * Special cases: NaN against NaN is 0; a reference beyond the binary32 range
 * counts as 0 when y is the infinity of its sign (and as a huge error
 * otherwise); a zero reference requires a zero of the same sign.
 */
#include <dlfcn.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <string.h>

typedef float (*f32_fn)(float);
typedef double (*f64_fn)(double);

struct job {
  f32_fn f;
  f64_fn g;
  uint64_t lo, hi;      /* bit patterns [lo, hi) */
  double max_err;
  uint32_t argmax;
  uint64_t bad_special;
};

static double ulp_err(float y, double r) {
  if (isnan(r)) return isnan(y) ? 0.0 : INFINITY;
  if (isnan(y)) return INFINITY;
  if (isinf(r) || fabs(r) >= 0x1.ffffffp127) {          /* beyond FLT_MAX + half an ulp */
    return (isinf(y) && !signbit(y) == !signbit(r)) ? 0.0 : INFINITY;
  }
  if (r == 0.0) return (y == 0.0f && !signbit(y) == !signbit(r)) ? 0.0 : INFINITY;
  int e = ilogb(r);
  if (e < -126) e = -126;
  return fabs((double)y - r) / ldexp(1.0, e - 23);
}

static void *run(void *p) {
  struct job *j = (struct job *)p;
  double mx = 0;
  uint32_t am = 0;
  for (uint64_t b = j->lo; b < j->hi; b++) {
    uint32_t u = (uint32_t)b;
    float x;
    memcpy(&x, &u, 4);
    double e = ulp_err(j->f(x), j->g((double)x));
    if (e > mx) { mx = e; am = u; }
  }
  j->max_err = mx;
  j->argmax = am;
  return NULL;
}

/* max ulp error of f32_name against f64_name over patterns [lo, hi), with
 * nthreads threads; *argmax receives the worst input's bits */
double exhaustive_max_ulp(const char *lib, const char *f32_name, const char *f64_name, uint64_t lo, uint64_t hi,
                          int nthreads, uint32_t *argmax) {
  void *h = dlopen(lib, RTLD_NOW | RTLD_LOCAL);
  if (!h) return -1.0;
  f32_fn f = (f32_fn)dlsym(h, f32_name);
  f64_fn g = (f64_fn)dlsym(h, f64_name);
  if (!f || !g || nthreads < 1 || nthreads > 256) return -2.0;
  struct job jobs[256];
  pthread_t th[256];
  uint64_t span = (hi - lo + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    jobs[t].f = f;
    jobs[t].g = g;
    jobs[t].lo = lo + t * span < hi ? lo + t * span : hi;
    jobs[t].hi = lo + (t + 1) * span < hi ? lo + (t + 1) * span : hi;
    pthread_create(&th[t], NULL, run, &jobs[t]);
  }
  double mx = 0;
  uint32_t am = 0;
  for (int t = 0; t < nthreads; t++) {
    pthread_join(th[t], NULL);
    if (jobs[t].max_err > mx) { mx = jobs[t].max_err; am = jobs[t].argmax; }
  }
  *argmax = am;
  return mx;
}
