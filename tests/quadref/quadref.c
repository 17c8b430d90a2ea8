/*
 * __float128 (libquadmath) reference values and ULP errors: the plain
 * definitions the oracle is pinned to.  Test-only; x86-64 (gcc's
 * __float128 with libquadmath).
 *
 * ULP definition (the paper measures "error in ULP" against MPFR in
 * Section 6 without a formula; this reading): for a reference value ref,
 * ulp(ref) = 2^(max(floor(log2|ref|), emin) - p + 1), p = 53 / 24,
 * emin = -1022 / -126.  If ref rounds to infinity in the target format, an
 * infinity of the right sign has error 0.  NaN against NaN is 0.  A zero
 * reference must be matched by a zero of the same sign.
 */
#include <quadmath.h>
#include <math.h>
#include <string.h>
#include <stdint.h>
#include <stddef.h>

typedef __float128 Q;

static Q q_pow(Q x, Q y) { return powq(x, y); }

/* reference value of fn at (x, y) */
static int eval(const char *fn, double xd, double yd, Q *r) {
  Q x = xd, y = yd;
  if (!strcmp(fn, "sin")) *r = sinq(x);
  else if (!strcmp(fn, "cos")) *r = cosq(x);
  else if (!strcmp(fn, "tan")) *r = tanq(x);
  else if (!strcmp(fn, "asin")) *r = asinq(x);
  else if (!strcmp(fn, "acos")) *r = acosq(x);
  else if (!strcmp(fn, "atan")) *r = atanq(x);
  else if (!strcmp(fn, "atan2")) *r = atan2q(x, y);
  else if (!strcmp(fn, "exp")) *r = expq(x);
  else if (!strcmp(fn, "exp2")) *r = exp2q(x);
  else if (!strcmp(fn, "exp10")) *r = powq((Q)10, x);
  else if (!strcmp(fn, "expm1")) *r = expm1q(x);
  else if (!strcmp(fn, "log")) *r = logq(x);
  else if (!strcmp(fn, "log2")) *r = log2q(x);
  else if (!strcmp(fn, "log10")) *r = log10q(x);
  else if (!strcmp(fn, "log1p")) *r = log1pq(x);
  else if (!strcmp(fn, "pow")) *r = q_pow(x, y);
  else if (!strcmp(fn, "cbrt")) *r = cbrtq(x);
  else if (!strcmp(fn, "sinh")) *r = sinhq(x);
  else if (!strcmp(fn, "cosh")) *r = coshq(x);
  else if (!strcmp(fn, "tanh")) *r = tanhq(x);
  else if (!strcmp(fn, "asinh")) *r = asinhq(x);
  else if (!strcmp(fn, "acosh")) *r = acoshq(x);
  else if (!strcmp(fn, "atanh")) *r = atanhq(x);
  else if (!strcmp(fn, "erf")) *r = erfq(x);
  else if (!strcmp(fn, "erfc")) *r = erfcq(x);
  else if (!strcmp(fn, "tgamma")) *r = tgammaq(x);
  else if (!strcmp(fn, "lgamma")) *r = lgammaq(x);
  else if (!strcmp(fn, "fmod")) *r = fmodq(x, y);
  else if (!strcmp(fn, "remainder")) *r = remainderq(x, y);
  else if (!strcmp(fn, "hypot")) *r = hypotq(x, y);
  else if (!strcmp(fn, "sqrt")) *r = sqrtq(x);
  else if (!strcmp(fn, "sinpi") || !strcmp(fn, "cospi")) {
    /* reduce exactly in binary128 (x is a double): r = x - 2 rint(x/2) in [-1, 1] */
    if (isinfq(x) || isnanq(x)) { *r = nanq(""); return 0; }
    Q rr = x - 2 * rintq(x / 2);
    if (!strcmp(fn, "sinpi")) {
      if (rr == rintq(rr)) { *r = signbitq(x) ? -(Q)0 : (Q)0; return 0; }   /* integers: +-0 */
      if (rr > 0.5Q) rr = 1 - rr;                    /* sin(pi r) = sin(pi (1 - r)) */
      if (rr < -0.5Q) rr = -1 - rr;
      *r = sinq(M_PIq * rr);
    } else {
      Q h = 0.5Q - fabsq(rr);                        /* cos(pi r) = sin(pi (1/2 - |r|)) */
      *r = h == 0 ? (Q)0 : sinq(M_PIq * h);
    }
  }
  else return -1;
  return 0;
}

static double ulp_err(Q ref, double out, int p, int emin, int emax) {
  if (isnanq(ref)) return isnan(out) ? 0.0 : INFINITY;
  if (isnan(out)) return INFINITY;
  /* values at or above max + ulp(max)/2 round to infinity */
  Q thr = ldexpq((Q)1, emax + 1) - ldexpq((Q)1, emax - p);
  if (isinfq(ref) || fabsq(ref) >= thr) {
    if (isinf(out) && ((out > 0) == (ref > 0))) return 0.0;
    if (isinfq(ref)) return INFINITY;
  }
  if (ref == 0) {
    if (out != 0) return INFINITY;
    return (signbit(out) != 0) == (signbitq(ref) != 0) ? 0.0 : INFINITY;
  }
  if (isinf(out)) return INFINITY;
  int e;
  frexpq(ref, &e);           /* |ref| in [2^(e-1), 2^e) */
  int lg = e - 1;
  if (lg < emin) lg = emin;
  Q ulp = ldexpq((Q)1, lg - p + 1);
  return (double)(fabsq((Q)out - ref) / ulp);
}

/* err[i] = ULP error of out[i] against fn(x[i], y[i]) in binary64 */
int quad_ulp_f64(const char *fn, const double *x, const double *y, const double *out,
                 double *err, size_t n) {
  for (size_t i = 0; i < n; i++) {
    Q r;
    if (eval(fn, x[i], y ? y[i] : 0.0, &r)) return -1;
    err[i] = ulp_err(r, out[i], 53, -1022, 1023);
  }
  return 0;
}

/* the same in binary32 (inputs and outputs are floats) */
int quad_ulp_f32(const char *fn, const float *x, const float *y, const float *out,
                 double *err, size_t n) {
  for (size_t i = 0; i < n; i++) {
    Q r;
    if (eval(fn, x[i], y ? y[i] : 0.0f, &r)) return -1;
    err[i] = ulp_err(r, out[i], 24, -126, 127);
  }
  return 0;
}

/* reference rounded to double (RN), for cross-checks against the host libm */
int quad_ref_f64(const char *fn, const double *x, const double *y, double *out, size_t n) {
  for (size_t i = 0; i < n; i++) {
    Q r;
    if (eval(fn, x[i], y ? y[i] : 0.0, &r)) return -1;
    out[i] = (double)r;
  }
  return 0;
}

/* err[i] = ULP error of out[i] (given as a double) in a format with p-bit
 * significands and exponent range [emin, emax] (bf16: 8, -126, 127; binary16:
 * 11, -14, 15), inputs given as doubles */
int quad_ulp_gen(const char *fn, const double *x, const double *out, double *err, size_t n,
                 int p, int emin, int emax) {
  for (size_t i = 0; i < n; i++) {
    Q r;
    if (eval(fn, x[i], 0.0, &r)) return -1;
    err[i] = ulp_err(r, out[i], p, emin, emax);
  }
  return 0;
}
