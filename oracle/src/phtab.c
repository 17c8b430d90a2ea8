/*
 * Payne-Hanek table of the oracle, computed at load time with a small
 * fixed-point bignum (no MPFR: only its runtime library exists here).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 *
 * Section 5.8 and Appendix A (the Payne-Hanek table-generation figure):
 *   for E = 0..1023, with M = (E > 700 ? -128 : 0),
 *   m = frac(2/pi * 2^(E-53)) * 2^-(E-53+M),
 *   four times: t = RN_double(m) with its lowest bit cleared; tab[4E+i] = t; m -= t.
 * The figure works at 1280 bits; this generator keeps FRAC_BITS fractional
 * bits, more than the 970-bit shift plus the 4 x 53 stored bits need.
 *
 * In addition (reading of Section 5.8 for a full-turn reduction), ibit[E] is
 * the parity of I(E) = floor(2/pi * 2^(E-53)); the table drops M*I(E)/2
 * turns, which is a half turn exactly when the mantissa M and I(E) are odd.
 *
 * pi comes from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239) evaluated
 * in fixed point; 2/pi is then a bit-by-bit long division.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define FRAC_LIMBS 56                 /* 1792 fractional bits */
#define INT_LIMBS 2
#define NL (FRAC_LIMBS + INT_LIMBS)
#define FRAC_BITS (32 * FRAC_LIMBS)

typedef struct { uint32_t w[NL]; } big;   /* little-endian limbs; value = N / 2^FRAC_BITS */

static void b_zero(big *a) { memset(a, 0, sizeof *a); }
static int b_iszero(const big *a) { for (int i = 0; i < NL; i++) if (a->w[i]) return 0; return 1; }
static void b_add(big *r, const big *a, const big *b) {
  uint64_t c = 0;
  for (int i = 0; i < NL; i++) { c += (uint64_t)a->w[i] + b->w[i]; r->w[i] = (uint32_t)c; c >>= 32; }
}
static void b_sub(big *r, const big *a, const big *b) {   /* requires a >= b */
  int64_t br = 0;
  for (int i = 0; i < NL; i++) {
    int64_t d = (int64_t)a->w[i] - b->w[i] - br;
    br = d < 0; r->w[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
  }
}
static int b_cmp(const big *a, const big *b) {
  for (int i = NL - 1; i >= 0; i--) if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  return 0;
}
static void b_divs(big *a, uint32_t d) {   /* a /= d, truncating */
  uint64_t r = 0;
  for (int i = NL - 1; i >= 0; i--) { uint64_t c = (r << 32) | a->w[i]; a->w[i] = (uint32_t)(c / d); r = c % d; }
}
static void b_muls(big *a, uint32_t m) {
  uint64_t c = 0;
  for (int i = 0; i < NL; i++) { c += (uint64_t)a->w[i] * m; a->w[i] = (uint32_t)c; c >>= 32; }
}
static void b_shl1(big *a) {
  for (int i = NL - 1; i > 0; i--) a->w[i] = (a->w[i] << 1) | (a->w[i - 1] >> 31);
  a->w[0] <<= 1;
}
static int b_bit(const big *a, int k) { return (k < 0 || k >= 32 * NL) ? 0 : (a->w[k >> 5] >> (k & 31)) & 1; }
static void b_setbit(big *a, int k) { a->w[k >> 5] |= 1u << (k & 31); }
static int b_topbit(const big *a) {
  for (int i = NL - 1; i >= 0; i--) if (a->w[i]) return 32 * i + 31 - __builtin_clz(a->w[i]);
  return -1;
}

/* atan(1/k) * 2^FRAC_BITS by its Taylor series */
static void b_atan_inv(big *r, uint32_t k) {
  big t, term; b_zero(r); b_zero(&t);
  t.w[FRAC_LIMBS] = 1;             /* 1.0 */
  b_divs(&t, k);                   /* 1/k */
  for (uint32_t n = 0; !b_iszero(&t); n++) {
    term = t; b_divs(&term, 2 * n + 1);
    if (n & 1) b_sub(r, r, &term); else b_add(r, r, &term);
    b_divs(&t, k); b_divs(&t, k);
  }
}

static double tab[4096];
static uint8_t ibit[1024];
static float tabf[512];
static uint8_t ibitf[128];
static int ready;

/* round the (non-negative) fixed-point value v * 2^scale to a binary
 * floating-point number with p-bit significands and smallest exponent
 * emin_sub of its subnormals (53/-1074 double, 24/-149 float), RN-even;
 * returns 0 for v == 0 */
static double b_round(const big *v, int scale, int p, int emin_sub) {
  int tb = b_topbit(v);
  if (tb < 0) return 0.0;
  int e = tb - FRAC_BITS + scale;                 /* ilogb of the value */
  int ulpe = e - (p - 1) < emin_sub ? emin_sub : e - (p - 1);   /* exponent of the last kept bit */
  int lo = ulpe - scale + FRAC_BITS;              /* bit index of the last kept bit */
  uint64_t m = 0;
  for (int k = tb; k >= lo; k--) m = (m << 1) | (uint64_t)b_bit(v, k);
  int half = b_bit(v, lo - 1), sticky = 0;
  for (int k = lo - 2; k >= 0 && !sticky; k--) sticky = b_bit(v, k);
  if (half && (sticky || (m & 1))) m++;
  return ldexp((double)m, ulpe);
}
static double b_to_double(const big *v, int scale) { return b_round(v, scale, 53, -1074); }

/* the exact fixed-point value of |t| * 2^-scale (t a double) */
static void b_from_double(big *r, double t, int scale) {
  b_zero(r);
  int e; double fr = frexp(fabs(t), &e);          /* |t| = fr * 2^e, fr in [0.5,1) */
  uint64_t m = (uint64_t)ldexp(fr, 53);
  int base = e - 53 - scale + FRAC_BITS;          /* bit index of m's lowest bit */
  for (int k = 0; k < 53; k++) if ((m >> k) & 1) b_setbit(r, base + k);
}

static void build(void) {
  big a, b, pi, two_over_pi, rem;
  b_atan_inv(&a, 5); b_muls(&a, 16);
  b_atan_inv(&b, 239); b_muls(&b, 4);
  b_sub(&pi, &a, &b);
  /* 2/pi = floor(2^(2F+1) / (pi 2^F)) / 2^F by restoring long division */
  b_zero(&two_over_pi); b_zero(&rem);
  for (int i = 2 * FRAC_BITS + 1; i >= 0; i--) {
    b_shl1(&rem);
    if (i == 2 * FRAC_BITS + 1) rem.w[0] |= 1;
    if (b_cmp(&rem, &pi) >= 0) { b_sub(&rem, &rem, &pi); if (i < 32 * NL) b_setbit(&two_over_pi, i); }
  }
  for (int E = 0; E < 1024; E++) {
    int sh = E - 53, M = E > 700 ? -128 : 0;
    big fr; b_zero(&fr);
    /* fr = frac(2/pi * 2^sh) in fixed point */
    for (int k = 0; k < FRAC_BITS; k++) if (b_bit(&two_over_pi, k - sh)) b_setbit(&fr, k);
    ibit[E] = (uint8_t)(sh >= 0 ? b_bit(&two_over_pi, FRAC_BITS - sh) : 0);
    int scale = -(E - 53 + M);
    int neg = 0;                                  /* sign of the running remainder */
    for (int i = 0; i < 4; i++) {
      double t = b_to_double(&fr, scale);
      uint64_t bits; memcpy(&bits, &t, 8); bits &= ~(uint64_t)1; memcpy(&t, &bits, 8);
      tab[4 * E + i] = neg ? -t : t;
      big tv; b_from_double(&tv, t, scale);
      if (b_cmp(&fr, &tv) >= 0) b_sub(&fr, &fr, &tv);
      else { b_sub(&fr, &tv, &fr); neg = !neg; }
    }
  }
  /* FP32 table: the same definition with 24-bit words, E = 0..127,
   * M = (E > 64 ? -64 : 0), m = frac(2/pi 2^(E-24)) 2^-(E-24+M) */
  for (int E = 0; E < 128; E++) {
    int sh = E - 24, M = E > 64 ? -64 : 0;
    big fr; b_zero(&fr);
    for (int k = 0; k < FRAC_BITS; k++) if (b_bit(&two_over_pi, k - sh)) b_setbit(&fr, k);
    ibitf[E] = (uint8_t)(sh >= 0 ? b_bit(&two_over_pi, FRAC_BITS - sh) : 0);
    int scale = -(E - 24 + M);
    int neg = 0;
    for (int i = 0; i < 4; i++) {
      float t = (float)b_round(&fr, scale, 24, -149);     /* exact: already 24 bits */
      uint32_t bits; memcpy(&bits, &t, 4); bits &= ~(uint32_t)1; memcpy(&t, &bits, 4);
      tabf[4 * E + i] = neg ? -t : t;
      big tv; b_from_double(&tv, (double)t, scale);
      if (b_cmp(&fr, &tv) >= 0) b_sub(&fr, &fr, &tv);
      else { b_sub(&fr, &tv, &fr); neg = !neg; }
    }
  }
  ready = 1;
}

__attribute__((constructor)) static void init_tables(void) { if (!ready) build(); }

const double *oracle_ph_tab(void) { if (!ready) build(); return tab; }
const uint8_t *oracle_ph_ibit(void) { if (!ready) build(); return ibit; }

const float *oracle_ph_tabf(void) { if (!ready) build(); return tabf; }
const uint8_t *oracle_ph_ibitf(void) { if (!ready) build(); return ibitf; }

void oracle_ph_tablef_copy(float *out512, uint8_t *ibit128) {
  if (!ready) build();
  memcpy(out512, tabf, sizeof tabf);
  memcpy(ibit128, ibitf, sizeof ibitf);
}

void oracle_ph_table_copy(double *out4096, uint8_t *ibit1024) {
  if (!ready) build();
  memcpy(out4096, tab, sizeof tab);
  memcpy(ibit1024, ibit, sizeof ibit);
}
