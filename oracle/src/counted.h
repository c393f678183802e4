// Oracle: an operation-counting scalar type.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Counted wraps a double and counts, per thread, the floating-point
// operations applied to it: additions and subtractions, multiplications,
// divisions, square roots (each one operation) and evaluations of special
// functions (log, exp, sin, cos, pow: counted apart, they are not FLOP).
// Negation, comparisons, fabs, fmin and fmax are not counted.  Instantiating
// the oracle's templated routines with Counted gives the algorithmic
// operation count of what they compute.
#pragma once
#include <cmath>
#include <cstdint>

namespace orc {

struct OpCounts {
  int64_t add = 0, mul = 0, div = 0, sqrt = 0, fn = 0;
  int64_t flop() const { return add + mul + div + sqrt; }
};
inline thread_local OpCounts g_ops;

struct Counted {
  double v = 0.0;
  Counted() = default;
  Counted(double x) : v(x) {}  // constants enter without a count
};

inline Counted operator+(Counted a, Counted b) { ++g_ops.add; return a.v + b.v; }
inline Counted operator-(Counted a, Counted b) { ++g_ops.add; return a.v - b.v; }
inline Counted operator*(Counted a, Counted b) { ++g_ops.mul; return a.v * b.v; }
inline Counted operator/(Counted a, Counted b) { ++g_ops.div; return a.v / b.v; }
inline Counted operator-(Counted a) { return -a.v; }
inline Counted& operator+=(Counted& a, Counted b) { return a = a + b; }
inline Counted& operator-=(Counted& a, Counted b) { return a = a - b; }
inline Counted& operator*=(Counted& a, Counted b) { return a = a * b; }
inline Counted& operator/=(Counted& a, Counted b) { return a = a / b; }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { return a.v != b.v; }

inline Counted sqrt(Counted a) { ++g_ops.sqrt; return std::sqrt(a.v); }
inline Counted log(Counted a) { ++g_ops.fn; return std::log(a.v); }
inline Counted exp(Counted a) { ++g_ops.fn; return std::exp(a.v); }
inline Counted sin(Counted a) { ++g_ops.fn; return std::sin(a.v); }
inline Counted cos(Counted a) { ++g_ops.fn; return std::cos(a.v); }
inline Counted pow(Counted a, Counted b) { ++g_ops.fn; return std::pow(a.v, b.v); }
inline Counted fabs(Counted a) { return std::fabs(a.v); }
inline Counted fmax(Counted a, Counted b) { return std::fmax(a.v, b.v); }
inline double value(Counted a) { return a.v; }
inline double value(double a) { return a; }

}  // namespace orc
