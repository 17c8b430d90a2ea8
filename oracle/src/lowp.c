/*
 * bf16 / f16 forms of the oracle: convert the 16-bit input to binary32
 * (exact), evaluate the FP32 oracle function, round the result to the 16-bit
 * format (round-to-nearest-even); NaN results are the canonical quiet NaN of
 * the format (0x7FC0 bf16, 0x7E00 f16).
 *
 * Test infrastructure: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark use anything under oracle/.
 */
#include "oracle.h"

static float bf16_to_f32(uint16_t h) { uint32_t b = (uint32_t)h << 16; float f; memcpy(&f, &b, 4); return f; }
static uint16_t f32_to_bf16(float f) {
  uint32_t b = fbits(f);
  if ((b & 0x7FFFFFFFu) > 0x7F800000u) return 0x7FC0;
  b += 0x7FFFu + ((b >> 16) & 1u);           /* round to nearest, ties to even */
  return (uint16_t)(b >> 16);
}
static float f16_to_f32(uint16_t h) {
  uint32_t s = (uint32_t)(h & 0x8000u) << 16, e = (h >> 10) & 0x1F, m = h & 0x3FFu, b;
  if (e == 0x1F) b = s | 0x7F800000u | (m << 13);
  else if (e) b = s | ((e + 112) << 23) | (m << 13);
  else {                                       /* subnormal: m * 2^-24, exact in binary32 */
    float f = (float)m * 0x1p-24f;
    return s ? -f : f;
  }
  float f; memcpy(&f, &b, 4); return f;
}
static uint16_t f32_to_f16(float f) {
  uint32_t b = fbits(f), sign = (b >> 16) & 0x8000u, ab = b & 0x7FFFFFFFu;
  if (ab > 0x7F800000u) return 0x7E00;
  if (ab >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u);        /* >= 65520: inf */
  if (ab >= 0x38800000u) {                                         /* normal half */
    uint32_t r = ab - (112u << 23);
    r += 0xFFFu + ((r >> 13) & 1u);
    return (uint16_t)(sign | (r >> 13));
  }
  /* subnormal half: |f| + 0.5 rounds |f| to a multiple of 2^-24 (ties to even) */
  float a; memcpy(&a, &ab, 4);
  uint32_t t = fbits(a + 0.5f) - 0x3F000000u;
  return (uint16_t)(sign | t);
}

#define LOWP(FN, ACC)                                                                   \
  uint16_t oracle_##FN##_##ACC##_bf16(uint16_t h) {                                     \
    return f32_to_bf16(oracle_##FN##_##ACC##_f32(bf16_to_f32(h)));                      \
  }                                                                                     \
  uint16_t oracle_##FN##_##ACC##_f16(uint16_t h) {                                      \
    return f32_to_f16(oracle_##FN##_##ACC##_f32(f16_to_f32(h)));                        \
  }
LOWP(erf, u10) LOWP(erf, u35) LOWP(tanh, u10) LOWP(tanh, u35)
LOWP(exp, u10) LOWP(exp, u35) LOWP(log1p, u10) LOWP(log1p, u35)

/* conversions exported for the pins */
float oracle_bf16_to_f32(uint16_t h) { return bf16_to_f32(h); }
uint16_t oracle_f32_to_bf16(float f) { return f32_to_bf16(f); }
float oracle_f16_to_f32(uint16_t h) { return f16_to_f32(h); }
uint16_t oracle_f32_to_f16(float f) { return f32_to_f16(f); }
