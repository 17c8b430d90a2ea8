// FP32 sin and cos (u10, u35) in float-float arithmetic for sm_103a.
//
// Section 5.1 in binary32 only (no FP64): Cody-Waite with pi/2 split into
// three (|x| < 125) or four (|x| < 2^20) floats, the head by fmaf (exact in
// that range; an exact FF product for cos at |x| < 1, where it is not), the
// Payne-Hanek reduction of Section 5.8 in FF over the FP32 table (four 24-bit
// words per exponent, half-turn parity fix) above that; one sine polynomial
// on the half-turn grid, the leading products in FF for u10.
#include "trig32_core.cuh"

#ifndef SLEEFCU_FUNCTORS_ONLY
using namespace sleefcu;

// binary32: the plain grid-stride kernel (a measured 3-15 % faster here than the
// divergence-sorted one, whose bookkeeping costs about what it saves when every
// operation is a cheap binary32 one)
#define SORTED32(NAME, F)                                                                   \
  extern "C" sleefcu_status sleefcu_##NAME(const float *x, float *out, size_t n,            \
                                           sleefcu_stream s) {                              \
    return launch_unary32<trig32::F>("sleefcu_" #NAME, x, out, n, s);                       \
  }
SORTED32(sin_u10_f32, SinU10)
SORTED32(sin_u35_f32, SinU35)
SORTED32(cos_u10_f32, CosU10)
SORTED32(cos_u35_f32, CosU35)
#undef SORTED32
#endif  // SLEEFCU_FUNCTORS_ONLY
