// Host-side checks of the software binary64 arithmetic (softfp64.cuh, the
// header the kernels use) against the host processor's IEEE operations:
// fma() from the C library, +, *, rint() and trunc() in the default rounding mode
// (round to nearest, ties to even).  Test infrastructure, built by
// tests/test_softfp.py with g++.
#include <math.h>

#include "softfp_gen.h"

static bool same(uint64_t got, uint64_t want) { return is_nan(want) ? is_nan(got) : got == want; }

extern "C" {

// n random triples per mode of mode_mask (bit k: mode k); compares fma, add
// (a + c), mul (a b), rint (a) and trunc (b); returns the number of
// mismatches and the first one in bad[0..4] (a, b, c, got, want) with bad[5]
// = the operation (0 fma, 1 add, 2 mul, 3 rint, 4 trunc)
int64_t sfp_check(uint64_t seed, int64_t n, int mode_mask, uint64_t *bad) {
  Rng r{seed};
  int64_t errs = 0;
  for (int mode = 0; mode < 8; mode++) {
    if (!(mode_mask & (1 << mode))) continue;
    for (int64_t i = 0; i < n; i++) {
      uint64_t a, b, c;
      gen(r, mode, a, b, c);
      uint64_t got[5] = {S::fma(a, b, c), S::add(a, c), S::mul(a, b), S::rint(a), S::trunc(b)};
      uint64_t want[5] = {b_of(fma(d_of(a), d_of(b), d_of(c))), b_of(d_of(a) + d_of(c)),
                          b_of(d_of(a) * d_of(b)), b_of(rint(d_of(a))), b_of(trunc(d_of(b)))};
      for (int op = 0; op < 5; op++) {
        if (!same(got[op], want[op])) {
          if (errs == 0 && bad) {
            bad[0] = a; bad[1] = b; bad[2] = c; bad[3] = got[op]; bad[4] = want[op]; bad[5] = (uint64_t)op;
          }
          errs++;
        }
      }
    }
  }
  return errs;
}

// elementwise forms for directed cases
void sfp_fma_n(const uint64_t *a, const uint64_t *b, const uint64_t *c, uint64_t *out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = S::fma(a[i], b[i], c[i]);
}
void sfp_rint_n(const uint64_t *a, uint64_t *out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = S::rint(a[i]);
}
}

extern "C" {
// the host's own operations, for the directed cases
void ref_fma_n(const uint64_t *a, const uint64_t *b, const uint64_t *c, uint64_t *out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = b_of(fma(d_of(a[i]), d_of(b[i]), d_of(c[i])));
}
void ref_rint_n(const uint64_t *a, uint64_t *out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = b_of(rint(d_of(a[i])));
}
}
