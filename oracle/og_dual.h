/*
 * og_dual.h -- TEST INFRASTRUCTURE ONLY (see ebv_oracle.h).
 *
 * Forward-mode dual numbers v + d*e with e^2 = 0, for the oracle's own
 * derivatives: running the oracle's step with a parameter (or the body force)
 * seeded as x + 1*e gives the exact directional derivative of every result
 * in the e-part, with no truncation error.  The value part is computed by the
 * same operations in the same order as in plain double arithmetic, so it
 * equals the double run bit for bit.  Comparisons look at the value part
 * only: every branch (limiter, upwinding, the choice of a one-sided stencil)
 * takes the side the value takes, as a derivative of a piecewise smooth
 * function does away from its kinks.
 */
#ifndef OG_DUAL_H
#define OG_DUAL_H
#include <cmath>

struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double x) : v(x), d(0.0) {}  // NOLINT: constants enter as x + 0 e
    Dual(double x, double y) : v(x), d(y) {}
    Dual &operator+=(const Dual &b) { v += b.v; d += b.d; return *this; }
    Dual &operator-=(const Dual &b) { v -= b.v; d -= b.d; return *this; }
    Dual &operator*=(const Dual &b) { *this = Dual(v * b.v, d * b.v + v * b.d); return *this; }
    Dual &operator/=(const Dual &b) { *this = Dual(v / b.v, (d * b.v - v * b.d) / (b.v * b.v)); return *this; }
};

inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(const Dual &a, const Dual &b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual &a, const Dual &b)
{
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
inline bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
inline bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
inline bool operator==(const Dual &a, const Dual &b) { return a.v == b.v; }
inline bool operator!=(const Dual &a, const Dual &b) { return a.v != b.v; }

/* |x|: the derivative takes the sign of the value (+ at 0). */
inline Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }
/* sqrt: at 0 the derivative is taken as 0 (the strain-rate norm of a uniform
 * flow, where it is not differentiable). */
inline Dual sqrt(const Dual &a)
{
    double s = std::sqrt(a.v);
    return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual exp(const Dual &a)
{
    double e = std::exp(a.v);
    return Dual(e, a.d * e);
}
inline Dual expm1(const Dual &a) { return Dual(std::expm1(a.v), a.d * std::exp(a.v)); }
/* a^b; the b-part of the derivative only when b varies. */
inline Dual pow(const Dual &a, const Dual &b)
{
    double p = std::pow(a.v, b.v);
    double d = a.d != 0.0 ? a.d * b.v * std::pow(a.v, b.v - 1.0) : 0.0;
    if (b.d != 0.0) d += b.d * p * std::log(a.v);
    return Dual(p, d);
}

inline double value_of(double x) { return x; }
inline double value_of(const Dual &x) { return x.v; }
#endif
