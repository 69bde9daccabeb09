// Forward-mode dual numbers for the oracle (test infrastructure; not used by
// the CUDA path).
#pragma once

#include <cmath>

// ---------------------------------------------------------------------------
// forward-mode dual numbers with a fixed number of tangents
// ---------------------------------------------------------------------------
template <int NT>
struct Dual {
  double v;
  double d[NT];
  Dual() : v(0) { for (int i = 0; i < NT; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < NT; ++i) d[i] = 0; }
};
template <int NT> Dual<NT> operator+(const Dual<NT>& a, const Dual<NT>& b) { Dual<NT> r(a.v + b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int NT> Dual<NT> operator-(const Dual<NT>& a, const Dual<NT>& b) { Dual<NT> r(a.v - b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int NT> Dual<NT> operator-(const Dual<NT>& a) { Dual<NT> r(-a.v); for (int i = 0; i < NT; ++i) r.d[i] = -a.d[i]; return r; }
template <int NT> Dual<NT> operator*(const Dual<NT>& a, const Dual<NT>& b) { Dual<NT> r(a.v * b.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int NT> Dual<NT> operator/(const Dual<NT>& a, const Dual<NT>& b) { Dual<NT> r(a.v / b.v); for (int i = 0; i < NT; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v; return r; }
template <int NT> Dual<NT> operator+(const Dual<NT>& a, double b) { Dual<NT> r = a; r.v += b; return r; }
template <int NT> Dual<NT> operator+(double b, const Dual<NT>& a) { return a + b; }
template <int NT> Dual<NT> operator-(const Dual<NT>& a, double b) { Dual<NT> r = a; r.v -= b; return r; }
template <int NT> Dual<NT> operator-(double b, const Dual<NT>& a) { return -(a - b); }
template <int NT> Dual<NT> operator*(const Dual<NT>& a, double b) { Dual<NT> r(a.v * b); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b; return r; }
template <int NT> Dual<NT> operator*(double b, const Dual<NT>& a) { return a * b; }
template <int NT> Dual<NT> operator/(const Dual<NT>& a, double b) { return a * (1.0 / b); }
template <int NT> Dual<NT> operator/(double a, const Dual<NT>& b) { return Dual<NT>(a) / b; }
template <int NT> Dual<NT> dexp(const Dual<NT>& a) { double e = std::exp(a.v); Dual<NT> r(e); for (int i = 0; i < NT; ++i) r.d[i] = e * a.d[i]; return r; }
template <int NT> Dual<NT> dexpm1(const Dual<NT>& a) { double e = std::exp(a.v); Dual<NT> r(std::expm1(a.v)); for (int i = 0; i < NT; ++i) r.d[i] = e * a.d[i]; return r; }
template <int NT> Dual<NT> dsqrt(const Dual<NT>& a) { double r = std::sqrt(a.v); Dual<NT> o(r); for (int i = 0; i < NT; ++i) o.d[i] = (r > 0) ? a.d[i] / (2.0 * r) : 0.0; return o; }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dexp(double a) { return std::exp(a); }
inline double dexpm1(double a) { return std::expm1(a); }
template <int NT> double val(const Dual<NT>& a) { return a.v; }
inline double val(double a) { return a; }
