/*
 * Counting mode of the oracle (test infrastructure, like everything under
 * oracle/: only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark use it).
 *
 * The oracle's C sources are compiled a second time as C++ with this header
 * forced in first.  It replaces `double` and `float` by two classes that
 * hold one value of that type, perform every operation with the same single
 * IEEE round-to-nearest operation as the plain build (so every comparison,
 * select and loop trip comes out the same and each function takes the same
 * path), and add one to a per-thread tally for each floating-point
 * operation, by category:
 *
 *   ADD  add or subtract            MUL  multiply
 *   FMA  fused multiply-add         DIV  division
 *   SQRT square root                RND  rint / floor / ceil / trunc
 *   CMP  comparison                 CVT  conversion to an integer or to the
 *                                        other floating-point format
 *   SCL  ldexp / ilogb / frexp / nextafter (exponent or bit handling)
 *
 * Negation, fabs, copysign, isnan / isinf / isfinite / signbit and bit
 * copies are sign or bit operations and are not counted.  The algorithmic
 * operation count of a function (the roofline's unit of work for the
 * FP-pipe-bound kernels) is ADD + MUL + FMA + DIV + SQRT + RND; the other
 * categories are reported beside it.
 */
#ifndef ORACLE_OPCOUNT_HPP
#define ORACLE_OPCOUNT_HPP
#include <math.h>
#include <cmath>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

namespace opc {
enum { ADD, MUL, FMA, DIV, SQRT, RND, CMP, CVT, SCL, NCAT };
/* tally[0] counts binary64 operations, tally[1] binary32 operations */
extern thread_local uint64_t tally[2][NCAT];
inline void tick(int prec, int cat) { tally[prec][cat]++; }
}  // namespace opc

struct cf_t;

struct cd_t {
  double v;
  cd_t() = default;
  constexpr cd_t(double x) : v(x) {}
  constexpr cd_t(int x) : v(x) {}
  constexpr cd_t(unsigned x) : v(x) {}
  constexpr cd_t(long x) : v((double)x) {}
  constexpr cd_t(unsigned long x) : v((double)x) {}
  constexpr cd_t(long long x) : v((double)x) {}
  constexpr cd_t(unsigned long long x) : v((double)x) {}
  explicit cd_t(cf_t f);
  explicit operator int() const { opc::tick(0, opc::CVT); return (int)v; }
  explicit operator long() const { opc::tick(0, opc::CVT); return (long)v; }
  explicit operator long long() const { opc::tick(0, opc::CVT); return (long long)v; }
  explicit operator unsigned() const { opc::tick(0, opc::CVT); return (unsigned)v; }
  explicit operator unsigned long() const { opc::tick(0, opc::CVT); return (unsigned long)v; }
  explicit operator unsigned long long() const { opc::tick(0, opc::CVT); return (unsigned long long)v; }
  explicit operator bool() const { opc::tick(0, opc::CMP); return v != 0.0; }
  cd_t operator-() const { return cd_t(-v); }
  cd_t operator+() const { return *this; }
};

struct cf_t {
  float v;
  cf_t() = default;
  constexpr cf_t(float x) : v(x) {}
  /* explicit: a binary64 operand in binary32 code would make the plain build
   * compute that operation in binary64, so such an expression must not
   * compile here */
  explicit constexpr cf_t(double x) : v((float)x) {}
  constexpr cf_t(int x) : v((float)x) {}
  constexpr cf_t(unsigned x) : v((float)x) {}
  constexpr cf_t(long x) : v((float)x) {}
  constexpr cf_t(unsigned long x) : v((float)x) {}
  constexpr cf_t(long long x) : v((float)x) {}
  constexpr cf_t(unsigned long long x) : v((float)x) {}
  explicit cf_t(cd_t d) : v((float)d.v) { opc::tick(0, opc::CVT); }
  explicit operator int() const { opc::tick(1, opc::CVT); return (int)v; }
  explicit operator long() const { opc::tick(1, opc::CVT); return (long)v; }
  explicit operator long long() const { opc::tick(1, opc::CVT); return (long long)v; }
  explicit operator unsigned() const { opc::tick(1, opc::CVT); return (unsigned)v; }
  explicit operator unsigned long() const { opc::tick(1, opc::CVT); return (unsigned long)v; }
  explicit operator unsigned long long() const { opc::tick(1, opc::CVT); return (unsigned long long)v; }
  explicit operator bool() const { opc::tick(1, opc::CMP); return v != 0.0f; }
  cf_t operator-() const { return cf_t(-v); }
  cf_t operator+() const { return *this; }
};
inline cd_t::cd_t(cf_t f) : v((double)f.v) { opc::tick(1, opc::CVT); }

static_assert(sizeof(cd_t) == sizeof(double) && alignof(cd_t) == alignof(double), "cd_t layout");
static_assert(sizeof(cf_t) == sizeof(float) && alignof(cf_t) == alignof(float), "cf_t layout");

#define OPC_ARITH(T, P, R)                                                                      \
  inline T operator+(T a, T b) { opc::tick(P, opc::ADD); return T((R)(a.v + b.v)); }             \
  inline T operator-(T a, T b) { opc::tick(P, opc::ADD); return T((R)(a.v - b.v)); }             \
  inline T operator*(T a, T b) { opc::tick(P, opc::MUL); return T((R)(a.v * b.v)); }             \
  inline T operator/(T a, T b) { opc::tick(P, opc::DIV); return T((R)(a.v / b.v)); }             \
  inline T &operator+=(T &a, T b) { return a = a + b; }                                          \
  inline T &operator-=(T &a, T b) { return a = a - b; }                                          \
  inline T &operator*=(T &a, T b) { return a = a * b; }                                          \
  inline T &operator/=(T &a, T b) { return a = a / b; }                                          \
  inline bool operator<(T a, T b) { opc::tick(P, opc::CMP); return a.v < b.v; }                  \
  inline bool operator<=(T a, T b) { opc::tick(P, opc::CMP); return a.v <= b.v; }                \
  inline bool operator>(T a, T b) { opc::tick(P, opc::CMP); return a.v > b.v; }                  \
  inline bool operator>=(T a, T b) { opc::tick(P, opc::CMP); return a.v >= b.v; }                \
  inline bool operator==(T a, T b) { opc::tick(P, opc::CMP); return a.v == b.v; }                \
  inline bool operator!=(T a, T b) { opc::tick(P, opc::CMP); return a.v != b.v; }                \
  inline bool operator!(T a) { opc::tick(P, opc::CMP); return !(a.v != 0); }
OPC_ARITH(cd_t, 0, double)
OPC_ARITH(cf_t, 1, float)
#undef OPC_ARITH

/* binary64 math functions used by the oracle */
inline cd_t fma(cd_t a, cd_t b, cd_t c) { opc::tick(0, opc::FMA); return cd_t(std::fma(a.v, b.v, c.v)); }
inline cd_t sqrt(cd_t a) { opc::tick(0, opc::SQRT); return cd_t(std::sqrt(a.v)); }
inline cd_t rint(cd_t a) { opc::tick(0, opc::RND); return cd_t(std::rint(a.v)); }
inline cd_t floor(cd_t a) { opc::tick(0, opc::RND); return cd_t(std::floor(a.v)); }
inline cd_t ceil(cd_t a) { opc::tick(0, opc::RND); return cd_t(std::ceil(a.v)); }
inline cd_t trunc(cd_t a) { opc::tick(0, opc::RND); return cd_t(std::trunc(a.v)); }
inline cd_t fabs(cd_t a) { return cd_t(std::fabs(a.v)); }
inline cd_t copysign(cd_t a, cd_t b) { return cd_t(std::copysign(a.v, b.v)); }
inline bool isnan(cd_t a) { return std::isnan(a.v); }
inline bool isinf(cd_t a) { return std::isinf(a.v); }
inline bool isfinite(cd_t a) { return std::isfinite(a.v); }
inline bool signbit(cd_t a) { return std::signbit(a.v); }
inline cd_t ldexp(cd_t a, int e) { opc::tick(0, opc::SCL); return cd_t(std::ldexp(a.v, e)); }
inline int ilogb(cd_t a) { opc::tick(0, opc::SCL); return std::ilogb(a.v); }
inline cd_t frexp(cd_t a, int *e) { opc::tick(0, opc::SCL); return cd_t(std::frexp(a.v, e)); }
inline cd_t nextafter(cd_t a, cd_t b) { opc::tick(0, opc::SCL); return cd_t(std::nextafter(a.v, b.v)); }

/* binary32 math functions used by the oracle */
inline cf_t fmaf(cf_t a, cf_t b, cf_t c) { opc::tick(1, opc::FMA); return cf_t(std::fma(a.v, b.v, c.v)); }
inline cf_t sqrtf(cf_t a) { opc::tick(1, opc::SQRT); return cf_t(std::sqrt(a.v)); }
inline cf_t rintf(cf_t a) { opc::tick(1, opc::RND); return cf_t(std::rint(a.v)); }
inline cf_t floorf(cf_t a) { opc::tick(1, opc::RND); return cf_t(std::floor(a.v)); }
inline cf_t truncf(cf_t a) { opc::tick(1, opc::RND); return cf_t(std::trunc(a.v)); }
inline cf_t fabsf(cf_t a) { return cf_t(std::fabs(a.v)); }
inline cf_t copysignf(cf_t a, cf_t b) { return cf_t(std::copysign(a.v, b.v)); }
inline bool isnan(cf_t a) { return std::isnan(a.v); }
inline bool isinf(cf_t a) { return std::isinf(a.v); }
inline bool isfinite(cf_t a) { return std::isfinite(a.v); }
inline bool signbit(cf_t a) { return std::signbit(a.v); }
inline cf_t ldexpf(cf_t a, int e) { opc::tick(1, opc::SCL); return cf_t(std::ldexp(a.v, e)); }
inline int ilogbf(cf_t a) { opc::tick(1, opc::SCL); return std::ilogb(a.v); }
inline cf_t nextafterf(cf_t a, cf_t b) { opc::tick(1, opc::SCL); return cf_t(std::nextafter(a.v, b.v)); }

#define double cd_t
#define float cf_t
#endif
