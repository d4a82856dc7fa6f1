// Forward-mode (tangent) scalar: a value and its derivative with respect to
// one parameter.  The kinematics and the generated matrix elements are
// templated on their scalar types, so instantiating them with Dual<T>
// evaluates the integrand and its derivative in one pass, with the same
// operations as the value path.  Comparisons and branches use the value
// part only, so cut masks and interpolation cells are those of the base
// point (the pathwise derivative at fixed masks).
#pragma once
#include <cmath>

namespace mf {

// the float/double math functions stay visible next to the Dual overloads below
using ::fma;
using ::sqrt;
using ::exp;
using ::log;
using ::fabs;
using ::fmax;
using ::asinh;
using ::atan2;
#ifdef __CUDACC__
using ::sincospi;
#endif

template <typename T>
struct Dual {
    T v, d;
    Dual() = default;
    __host__ __device__ constexpr Dual(T value, T deriv) : v(value), d(deriv) {}
    __host__ __device__ constexpr Dual(double value) : v(T(value)), d(T(0)) {}
    __host__ __device__ constexpr Dual(float value) : v(T(value)), d(T(0)) {}
    __host__ __device__ constexpr Dual(int value) : v(T(value)), d(T(0)) {}
    template <typename U>
    __host__ __device__ explicit constexpr Dual(const Dual<U>& o) : v(T(o.v)), d(T(o.d)) {}
    __host__ __device__ Dual& operator+=(const Dual& o) { v += o.v; d += o.d; return *this; }
    __host__ __device__ Dual& operator-=(const Dual& o) { v -= o.v; d -= o.d; return *this; }
    __host__ __device__ Dual& operator*=(const Dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};

template <typename T> struct is_dual { static constexpr bool value = false; };
template <typename T> struct is_dual<Dual<T>> { static constexpr bool value = true; };

// the FP64 scalar that goes with a matrix-element type R: double for float and
// double, Dual<double> for Dual<float> and Dual<double>
template <typename R> struct Widen { using type = double; };
template <typename T> struct Widen<Dual<T>> { using type = Dual<double>; };
// a parameter of type T that takes no part in template argument deduction
template <typename T> struct NoDeduce { using type = T; };

// value part of a scalar
template <typename T> __host__ __device__ __forceinline__ T val(T x) { return x; }
template <typename T> __host__ __device__ __forceinline__ T val(const Dual<T>& x) { return x.v; }

template <typename T> __host__ __device__ __forceinline__ Dual<T> operator-(const Dual<T>& a) { return { -a.v, -a.d }; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return { a.v + b.v, a.d + b.d }; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return { a.v - b.v, a.d - b.d }; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> operator*(const Dual<T>& a, const Dual<T>& b)
{
    return { a.v * b.v, a.d * b.v + a.v * b.d };
}
template <typename T> __host__ __device__ __forceinline__ Dual<T> operator/(const Dual<T>& a, const Dual<T>& b)
{
    const T q = a.v / b.v;
    return { q, (a.d - q * b.d) / b.v };
}
#define MF_DUAL_MIXED(OP)                                                                                              \
    template <typename T> __host__ __device__ __forceinline__ Dual<T> operator OP(const Dual<T>& a, T b) { return a OP Dual<T>(b, T(0)); } \
    template <typename T> __host__ __device__ __forceinline__ Dual<T> operator OP(T a, const Dual<T>& b) { return Dual<T>(a, T(0)) OP b; }
MF_DUAL_MIXED(+)
MF_DUAL_MIXED(-)
MF_DUAL_MIXED(*)
MF_DUAL_MIXED(/)
#undef MF_DUAL_MIXED
#define MF_DUAL_CMP(OP)                                                                                                  \
    template <typename T> __host__ __device__ __forceinline__ bool operator OP(const Dual<T>& a, const Dual<T>& b) { return a.v OP b.v; } \
    template <typename T> __host__ __device__ __forceinline__ bool operator OP(const Dual<T>& a, T b) { return a.v OP b; }             \
    template <typename T> __host__ __device__ __forceinline__ bool operator OP(T a, const Dual<T>& b) { return a OP b.v; }
MF_DUAL_CMP(<)
MF_DUAL_CMP(>)
MF_DUAL_CMP(<=)
MF_DUAL_CMP(>=)
#undef MF_DUAL_CMP

template <typename T> __host__ __device__ __forceinline__ Dual<T> fma(const Dual<T>& a, const Dual<T>& b, const Dual<T>& c)
{
    return { fma(a.v, b.v, c.v), a.d * b.v + a.v * b.d + c.d };
}
template <typename T> __host__ __device__ __forceinline__ Dual<T> sqrt(const Dual<T>& a)
{
    const T s = sqrt(a.v);
    return { s, s > T(0) ? a.d / (T(2) * s) : T(0) };
}
template <typename T> __host__ __device__ __forceinline__ Dual<T> exp(const Dual<T>& a)
{
    const T e = exp(a.v);
    return { e, e * a.d };
}
template <typename T> __host__ __device__ __forceinline__ Dual<T> log(const Dual<T>& a) { return { log(a.v), a.d / a.v }; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> fabs(const Dual<T>& a) { return a.v < T(0) ? -a : a; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> fmax(const Dual<T>& a, const Dual<T>& b) { return a.v >= b.v ? a : b; }
template <typename T> __host__ __device__ __forceinline__ Dual<T> fmax(const Dual<T>& a, T b) { return a.v >= b ? a : Dual<T>(b, T(0)); }
template <typename T> __host__ __device__ __forceinline__ Dual<T> asinh(const Dual<T>& a)
{
    return { asinh(a.v), a.d / sqrt(a.v * a.v + T(1)) };
}
template <typename T> __host__ __device__ __forceinline__ Dual<T> atan2(const Dual<T>& y, const Dual<T>& x)
{
    const T r2 = x.v * x.v + y.v * y.v;
    return { atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2 };
}
#ifdef __CUDACC__
// sin and cos of pi a
template <typename T> __device__ __forceinline__ void sincospi(const Dual<T>& a, Dual<T>* s, Dual<T>* c)
{
    T sv, cv;
    sincospi(a.v, &sv, &cv);
    const T pi = T(3.14159265358979323846);
    *s = Dual<T>(sv, pi * cv * a.d);
    *c = Dual<T>(cv, -pi * sv * a.d);
}
#endif

}  // namespace mf
