/*
 * dual.h -- dual numbers (value, derivative) for forward-mode differentiation of the oracle.
 *
 * TEST INFRASTRUCTURE (part of the oracle). oracle_dual.cpp compiles the unchanged oracle.c with `double` meaning
 * `dual`, so the RHS, evaluated at u + eps*delta with eps^2 = 0, returns RHS(u) in .v and the directional
 * derivative J(u) delta in .d (the JVP), exact up to rounding. Each rule below is the derivative of the
 * elementary operation; comparisons use the value part.
 */
#pragma once
#include <math.h>

struct dual {
  double v, d;
  dual() : v(0.0), d(0.0) {}
  dual(double x) : v(x), d(0.0) {}  // NOLINT: implicit, constants are duals with zero derivative
  dual(long double x) : v((double)x), d(0.0) {}
  dual(int x) : v((double)x), d(0.0) {}
  dual(double x, double dx) : v(x), d(dx) {}
  explicit operator long double() const { return (long double)v; }
  explicit operator double() const { return v; }
  dual& operator+=(const dual& b) { v += b.v; d += b.d; return *this; }
  dual& operator-=(const dual& b) { v -= b.v; d -= b.d; return *this; }
  dual& operator*=(const dual& b) { *this = dual(v * b.v, d * b.v + v * b.d); return *this; }
  dual& operator/=(const dual& b) { *this = dual(v / b.v, (d * b.v - v * b.d) / (b.v * b.v)); return *this; }
};

inline dual operator+(const dual& a, const dual& b) { return dual(a.v + b.v, a.d + b.d); }
inline dual operator-(const dual& a, const dual& b) { return dual(a.v - b.v, a.d - b.d); }
inline dual operator-(const dual& a) { return dual(-a.v, -a.d); }
inline dual operator*(const dual& a, const dual& b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline dual operator/(const dual& a, const dual& b) { return dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline bool operator==(const dual& a, const dual& b) { return a.v == b.v; }
inline bool operator!=(const dual& a, const dual& b) { return a.v != b.v; }
inline bool operator<(const dual& a, const dual& b) { return a.v < b.v; }
inline bool operator>(const dual& a, const dual& b) { return a.v > b.v; }
inline bool operator<=(const dual& a, const dual& b) { return a.v <= b.v; }
inline bool operator>=(const dual& a, const dual& b) { return a.v >= b.v; }

inline dual log(const dual& a) { return dual(::log(a.v), a.d / a.v); }
inline dual log1p(const dual& a) { return dual(::log1p(a.v), a.d / (1.0 + a.v)); }
inline dual sqrt(const dual& a) {
  const double s = ::sqrt(a.v);
  return dual(s, a.d / (2.0 * s));
}
inline dual fabs(const dual& a) { return a.v < 0.0 ? -a : a; }
inline dual sin(const dual& a) { return dual(::sin(a.v), a.d * ::cos(a.v)); }
inline dual cos(const dual& a) { return dual(::cos(a.v), -a.d * ::sin(a.v)); }
