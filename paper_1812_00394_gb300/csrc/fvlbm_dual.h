// fvlbm_dual.h -- forward-mode (tangent) scalar for the FP64 tangent path of the library.
//
// Dual = value + derivative with respect to one parameter; arithmetic follows the chain rule.
// Instantiating the time-step kernels with this type gives the tangent-linear model of the
// discrete step (d f^{n+1} / dp from d f^n / dp and the seeded boundary / initial data).
// Non-smooth points take one-sided derivatives: comparisons, min / max and clips act on the
// value and carry the derivative of the selected branch; sqrt at exactly 0 has derivative 0.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define FVLBM_HD __host__ __device__
#else
#define FVLBM_HD
#endif

namespace fvlbm {

// The overloads below must not hide the plain floating-point ones inside this namespace.
using ::fmax;
using ::fmin;
using ::sqrt;
using ::tanh;

struct Dual {
    double v, d;
    FVLBM_HD Dual() : v(0), d(0) {}
    FVLBM_HD Dual(double x) : v(x), d(0) {}      // NOLINT: implicit from constants
    FVLBM_HD Dual(int x) : v(double(x)), d(0) {}  // NOLINT
    FVLBM_HD Dual(double x, double dx) : v(x), d(dx) {}
    FVLBM_HD explicit operator double() const { return v; }
    FVLBM_HD Dual &operator+=(const Dual &b) { v += b.v; d += b.d; return *this; }
    FVLBM_HD Dual &operator-=(const Dual &b) { v -= b.v; d -= b.d; return *this; }
    FVLBM_HD Dual &operator*=(const Dual &b) {
        d = d * b.v + v * b.d;
        v *= b.v;
        return *this;
    }
    FVLBM_HD Dual &operator/=(const Dual &b) {
        const double q = v / b.v;
        d = (d - q * b.d) / b.v;
        v = q;
        return *this;
    }
};

FVLBM_HD inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
FVLBM_HD inline Dual operator+(Dual a, const Dual &b) { return a += b; }
FVLBM_HD inline Dual operator-(Dual a, const Dual &b) { return a -= b; }
FVLBM_HD inline Dual operator*(Dual a, const Dual &b) { return a *= b; }
FVLBM_HD inline Dual operator/(Dual a, const Dual &b) { return a /= b; }
FVLBM_HD inline bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
FVLBM_HD inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
FVLBM_HD inline bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
FVLBM_HD inline bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
FVLBM_HD inline bool operator==(const Dual &a, const Dual &b) { return a.v == b.v; }
FVLBM_HD inline bool operator!=(const Dual &a, const Dual &b) { return a.v != b.v; }

FVLBM_HD inline Dual sqrt(const Dual &a) {
    const double s = ::sqrt(a.v);
    return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
FVLBM_HD inline Dual tanh(const Dual &a) {
    const double t = ::tanh(a.v);
    return Dual(t, a.d * (1.0 - t * t));
}
FVLBM_HD inline Dual fmin(const Dual &a, const Dual &b) { return b.v < a.v ? b : a; }
FVLBM_HD inline Dual fmax(const Dual &a, const Dual &b) { return b.v > a.v ? b : a; }

// Value and derivative parts: the plain floating types have derivative 0.
template <class T>
FVLBM_HD inline double value_of(const T &x) {
    return double(x);
}
FVLBM_HD inline double value_of(const Dual &x) { return x.v; }
template <class S>
FVLBM_HD inline S smin(const S &a, const S &b) {
    return b < a ? b : a;
}
template <class S>
FVLBM_HD inline S smax(const S &a, const S &b) {
    return b > a ? b : a;
}

// Derivative part of a value: 0 for the plain floating types.
template <class T>
FVLBM_HD inline double tangent_of(const T &) {
    return 0.0;
}
FVLBM_HD inline double tangent_of(const Dual &x) { return x.d; }

}  // namespace fvlbm
