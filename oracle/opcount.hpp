/*
 * opcount.hpp -- counting number type for the oracle's op-count mode.
 *
 * TEST INFRASTRUCTURE ONLY.  oracle/opcount.py compiles darts_oracle.c a
 * second time, as C++, with this header pre-included and ORC_OPCOUNT
 * defined.  Every `double` of the oracle then becomes orc_oc::D, a double
 * that tallies each arithmetic operation applied to it, so the counts are
 * those of the oracle's own plain restatement of the method (the paper's
 * equations in the order it states them), not a hand count.
 *
 * Tallies (one set per thread, reset per path by orc_opcount_paths):
 *   add   additions and subtractions (compound forms included)
 *   mul   multiplications
 *   div   divisions
 *   sqrt  square roots
 *   cmp   comparisons, min and max
 *   exp   exp, expm1
 *   log   log, log1p
 *   trig  sin, cos, tan, atan, atan2
 *   pow   pow
 *   philox  Philox4x32-10 blocks (integer work; 10 rounds each)
 * Negation, fabs and floor/ceil are not counted (a sign flip, a bit mask,
 * a conversion).  Operations on plain constants that never touch an
 * orc_oc::D are folded by the compiler and not counted either.
 */
#ifndef ORC_OPCOUNT_HPP
#define ORC_OPCOUNT_HPP

/* every system header the oracle includes, before `double` is redefined */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <type_traits>

typedef double orc_oc_plain;

namespace orc_oc {

enum { ADD, MUL, DIV, SQRT, CMP, EXP, LOG, TRIG, POW, PHILOX, N };

struct Tally {
  uint64_t n[N];
  int paused;
};
inline thread_local Tally tally = {};

inline void bump(int k) {
  if (!tally.paused) ++tally.n[k];
}

struct D {
  orc_oc_plain v;
  D() = default;
  D(orc_oc_plain x) : v(x) {}  // NOLINT: implicit, as a double would convert
  explicit operator orc_oc_plain() const { return v; }
  explicit operator float() const { return (float)v; }
  explicit operator int() const { return (int)v; }
  explicit operator unsigned() const { return (unsigned)v; }
  explicit operator long() const { return (long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned long long() const { return (unsigned long long)v; }
  explicit operator unsigned char() const { return (unsigned char)v; }
  D operator-() const { return D(-v); }
  D operator+() const { return *this; }
  D& operator+=(D o) { bump(ADD); v += o.v; return *this; }
  D& operator-=(D o) { bump(ADD); v -= o.v; return *this; }
  D& operator*=(D o) { bump(MUL); v *= o.v; return *this; }
  D& operator/=(D o) { bump(DIV); v /= o.v; return *this; }
};

template <class T>
using if_num = typename std::enable_if<std::is_arithmetic<T>::value, int>::type;

#define ORC_OC_BINOP(op, k)                                                              \
  inline D operator op(D a, D b) { bump(k); return D(a.v op b.v); }                     \
  template <class T, if_num<T> = 0>                                                      \
  inline D operator op(D a, T b) { bump(k); return D(a.v op (orc_oc_plain)b); }          \
  template <class T, if_num<T> = 0>                                                      \
  inline D operator op(T a, D b) { bump(k); return D((orc_oc_plain)a op b.v); }
ORC_OC_BINOP(+, ADD)
ORC_OC_BINOP(-, ADD)
ORC_OC_BINOP(*, MUL)
ORC_OC_BINOP(/, DIV)
#undef ORC_OC_BINOP

#define ORC_OC_CMP(op)                                                                   \
  inline bool operator op(D a, D b) { bump(CMP); return a.v op b.v; }                   \
  template <class T, if_num<T> = 0>                                                      \
  inline bool operator op(D a, T b) { bump(CMP); return a.v op (orc_oc_plain)b; }        \
  template <class T, if_num<T> = 0>                                                      \
  inline bool operator op(T a, D b) { bump(CMP); return (orc_oc_plain)a op b.v; }
ORC_OC_CMP(<)
ORC_OC_CMP(>)
ORC_OC_CMP(<=)
ORC_OC_CMP(>=)
ORC_OC_CMP(==)
ORC_OC_CMP(!=)
#undef ORC_OC_CMP

inline orc_oc_plain val(D a) { return a.v; }
template <class T, if_num<T> = 0>
inline orc_oc_plain val(T a) { return (orc_oc_plain)a; }

}  // namespace orc_oc

/* math functions of a counted value (global scope, as the C names are) */
#define ORC_OC_FN1(name, k)                                                              \
  inline orc_oc::D name(orc_oc::D a) { orc_oc::bump(orc_oc::k); return orc_oc::D(std::name(a.v)); }
ORC_OC_FN1(sqrt, SQRT)
ORC_OC_FN1(exp, EXP)
ORC_OC_FN1(expm1, EXP)
ORC_OC_FN1(log, LOG)
ORC_OC_FN1(log1p, LOG)
ORC_OC_FN1(log2, LOG)
ORC_OC_FN1(sin, TRIG)
ORC_OC_FN1(cos, TRIG)
ORC_OC_FN1(tan, TRIG)
ORC_OC_FN1(atan, TRIG)
#undef ORC_OC_FN1
inline orc_oc::D fabs(orc_oc::D a) { return orc_oc::D(std::fabs(a.v)); }
inline orc_oc::D floor(orc_oc::D a) { return orc_oc::D(std::floor(a.v)); }
inline orc_oc::D ceil(orc_oc::D a) { return orc_oc::D(std::ceil(a.v)); }
inline bool isfinite(orc_oc::D a) { return std::isfinite(a.v); }
inline bool isnan(orc_oc::D a) { return std::isnan(a.v); }
template <class A, class B>
inline orc_oc::D atan2(A a, B b) {
  orc_oc::bump(orc_oc::TRIG);
  return orc_oc::D(std::atan2(orc_oc::val(a), orc_oc::val(b)));
}
template <class A, class B>
inline orc_oc::D pow(A a, B b) {
  orc_oc::bump(orc_oc::POW);
  return orc_oc::D(std::pow(orc_oc::val(a), orc_oc::val(b)));
}
template <class A, class B>
inline orc_oc::D fmin(A a, B b) {
  orc_oc::bump(orc_oc::CMP);
  return orc_oc::D(std::fmin(orc_oc::val(a), orc_oc::val(b)));
}
template <class A, class B>
inline orc_oc::D fmax(A a, B b) {
  orc_oc::bump(orc_oc::CMP);
  return orc_oc::D(std::fmax(orc_oc::val(a), orc_oc::val(b)));
}

#define double orc_oc::D

#endif
