/*
 * counting.h -- an instrumented FP64 scalar for the oracle's flop count.
 *
 * TEST INFRASTRUCTURE.  With -DPF_ORACLE_COUNT, pf_oracle.c is compiled as
 * C++ with real_t = pf_count::Counting: every addition, subtraction,
 * multiplication, division and square root on the step's values is counted,
 * so one step over n sites gives the exact number of floating-point
 * operations per lattice update of the algorithm as the oracle writes it
 * (dense moment matrices, one site and one field at a time).  Operations on
 * plain doubles (constants, the initialisation) are not counted.  The value
 * itself is computed exactly as in the double build.
 */
#ifndef PF_ORACLE_COUNTING_H
#define PF_ORACLE_COUNTING_H
#include <cmath>

namespace pf_count {

struct Tally {
  unsigned long long add, mul, div, sqrt;
};
extern Tally g_tally;

struct Counting {
  double v;
  Counting() = default;
  Counting(double x) : v(x) {}
};

inline Counting operator+(Counting a, Counting b) { ++g_tally.add; return a.v + b.v; }
inline Counting operator-(Counting a, Counting b) { ++g_tally.add; return a.v - b.v; }
inline Counting operator*(Counting a, Counting b) { ++g_tally.mul; return a.v * b.v; }
inline Counting operator/(Counting a, Counting b) { ++g_tally.div; return a.v / b.v; }
inline Counting operator-(Counting a) { return -a.v; }
inline Counting& operator+=(Counting& a, Counting b) { a = a + b; return a; }
inline Counting& operator-=(Counting& a, Counting b) { a = a - b; return a; }
inline Counting& operator*=(Counting& a, Counting b) { a = a * b; return a; }
inline Counting& operator/=(Counting& a, Counting b) { a = a / b; return a; }
inline bool operator!=(Counting a, Counting b) { return a.v != b.v; }
inline bool operator==(Counting a, Counting b) { return a.v == b.v; }
inline Counting sqrt(Counting a) { ++g_tally.sqrt; return std::sqrt(a.v); }

}  // namespace pf_count

#endif
