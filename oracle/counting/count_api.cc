/*
 * Entry points of the counting build of the oracle (test infrastructure:
 * only tests/ use it).  Compiled as C++ with opcount.hpp forced in, so
 * `double` and `float` below are the counting types.
 *
 * oracle_count_apply(name, x, y, out, out2, n, tally) evaluates `name` over
 * n elements on the calling thread, like the plain build's oracle_apply,
 * and adds the operations it performed to tally[2][NCAT] (row 0 binary64,
 * row 1 binary32; column order ADD MUL FMA DIV SQRT RND CMP CVT SCL).
 * Returns 0, or -1 for an unknown name.
 *
 * oracle_count_ph(x, n, tally) runs the binary64 Payne-Hanek reduction of
 * Section 5.8 alone over n arguments (the operation count of the paper's
 * table comparing Payne-Hanek implementations).
 */
#include "oracle.h"

thread_local uint64_t opc::tally[2][opc::NCAT];

namespace {
enum { K_U64 = 1, K_B64 = 2, K_SC64 = 3, K_U32 = 11, K_B32 = 12, K_SC32 = 13, K_U16 = 21 };
struct entry {
  const char *name;
  int kind;
  void *f;
};
#define U64(n) { #n, K_U64, (void *)(double (*)(double))oracle_##n }
#define B64(n) { #n, K_B64, (void *)(double (*)(double, double))oracle_##n }
#define SC64(n) { #n, K_SC64, (void *)(void (*)(double, double *, double *))oracle_##n }
#define U32(n) { #n, K_U32, (void *)(float (*)(float))oracle_##n }
#define B32(n) { #n, K_B32, (void *)(float (*)(float, float))oracle_##n }
#define SC32(n) { #n, K_SC32, (void *)(void (*)(float, float *, float *))oracle_##n }
#define U16(n) { #n, K_U16, (void *)(uint16_t (*)(uint16_t))oracle_##n }
const entry REG[] = {
#include "registry.inc"
/* the C99 set: the floating-point kinds are counted; the int32 kinds
 * (ilogb, ldexp, frexp: exponent handling only) are not registered */
#define XU64(n) U64(n)
#define XB64(n) B64(n)
#define XSC64(n) SC64(n)
#define XU32(n) U32(n)
#define XB32(n) B32(n)
#define XSC32(n) SC32(n)
#define XUI64(n) { #n, 0, NULL }
#define XBI64(n) { #n, 0, NULL }
#define XSI64(n) { #n, 0, NULL }
#define XUI32(n) { #n, 0, NULL }
#define XBI32(n) { #n, 0, NULL }
#define XSI32(n) { #n, 0, NULL }
#include "registry_c99.inc"
  { nullptr, 0, nullptr }
};
const entry *find(const char *name) {
  for (const entry *e = REG; e->name; e++)
    if (!strcmp(e->name, name)) return e;
  return nullptr;
}
void take(uint64_t *out) {
  for (int p = 0; p < 2; p++)
    for (int c = 0; c < opc::NCAT; c++) {
      out[p * opc::NCAT + c] += opc::tally[p][c];
      opc::tally[p][c] = 0;
    }
}
void clear() { memset(opc::tally, 0, sizeof opc::tally); }
}  // namespace

extern "C" int oracle_count_ncat(void) { return opc::NCAT; }

extern "C" int oracle_count_apply(const char *name, const void *x, const void *y, void *out,
                                  void *out2, size_t n, uint64_t *tally) {
  const entry *e = find(name);
  if (!e) return -1;
  clear();
  for (size_t i = 0; i < n; i++) {
    switch (e->kind) {
      case K_U64: ((double *)out)[i] = ((double (*)(double))e->f)(((const double *)x)[i]); break;
      case K_B64:
        ((double *)out)[i] = ((double (*)(double, double))e->f)(((const double *)x)[i], ((const double *)y)[i]);
        break;
      case K_SC64:
        ((void (*)(double, double *, double *))e->f)(((const double *)x)[i], (double *)out + i, (double *)out2 + i);
        break;
      case K_U32: ((float *)out)[i] = ((float (*)(float))e->f)(((const float *)x)[i]); break;
      case K_B32:
        ((float *)out)[i] = ((float (*)(float, float))e->f)(((const float *)x)[i], ((const float *)y)[i]);
        break;
      case K_SC32:
        ((void (*)(float, float *, float *))e->f)(((const float *)x)[i], (float *)out + i, (float *)out2 + i);
        break;
      case K_U16: ((uint16_t *)out)[i] = ((uint16_t (*)(uint16_t))e->f)(((const uint16_t *)x)[i]); break;
    }
  }
  take(tally);
  return 0;
}

extern "C" void oracle_count_ph(const double *x, size_t n, uint64_t *tally) {
  clear();
  for (size_t i = 0; i < n; i++) {
    int q;
    (void)oracle_ph_reduce_dd(x[i], &q);
  }
  take(tally);
}
