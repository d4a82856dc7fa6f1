// Double-float arithmetic: a real number as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits computed on the FP32 pipes.  It carries the
// kinematics of the mixed-precision path, whose cancellations (conformal boost, PDF
// interpolation near x -> 1, propagator invariants of collinear pairs) need more than FP32
// but nowhere near FP64's 53 bits, on a GPU whose FP64 rate is 1/64 of its FP32 rate.
//
// Building blocks: the error-free transformations of a sum, TwoSum (Knuth, The Art of
// Computer Programming vol. 2, sec. 4.2.2) and Fast2Sum (Dekker, Numer. Math. 18 (1971)
// 224), and of a product with a fused multiply-add.  Sums, products and quotients follow
// the double-word algorithms of Joldes, Muller and Popescu, ACM TOMS 44 (2017) 4:1
// (accurate sum, relative error below 3u^2; product below 4u^2 (double-word operand) and
// 2u^2 (float operand); quotient below 15u^2, u = 2^-24).  The elementary functions are
// Taylor series after an argument reduction: exp by k ln 2 (ln 2 split in Cody and Waite's
// manner so that k times its head is exact) and five halvings undone in expm1 form, log by
// one Newton step on exp from the float logarithm of the reduced mantissa, sin and cos of
// pi a by quadrant.  Each is accurate to a few 1e-14 relative (absolute for log near 1),
// checked against the FP64 functions by the library's self-test entry point.  The exponent
// range is float's: below about 2e-31 in magnitude the tail is subnormal and the relative
// precision falls gradually towards float's.
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace mf {

// the float/double functions stay visible next to the double-float overloads below
using ::sqrt;
using ::exp;
using ::log;
using ::fabs;
#ifdef __CUDACC__
using ::sincospi;
#endif

struct Df {
    float hi, lo;
    Df() = default;
    __host__ __device__ constexpr Df(float h, float l) : hi(h), lo(l) {}
    // the nearest double-float of a double (compile-time constants fold to two floats)
    __host__ __device__ constexpr Df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit constexpr operator float() const { return hi + lo; }
    __host__ __device__ explicit constexpr operator double() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------------------ error-free transformations

#ifdef __CUDACC__

__device__ __forceinline__ Df df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return Df(s, e);
}
// |a| >= |b| (or a = 0)
__device__ __forceinline__ Df df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return Df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ Df df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return Df(p, __fmaf_rn(a, b, -p));
}

// ------------------------------------------------------------------ arithmetic

__device__ __forceinline__ Df df_add(const Df& x, const Df& y)
{
    const Df s = df_two_sum(x.hi, y.hi);
    const Df t = df_two_sum(x.lo, y.lo);
    const Df v = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ Df df_add(const Df& x, float y)
{
    const Df s = df_two_sum(x.hi, y);
    return df_fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
__device__ __forceinline__ Df df_mul(const Df& x, const Df& y)
{
    const Df c = df_two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo)));
    return df_fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}
__device__ __forceinline__ Df df_mul(const Df& x, float y)
{
    const Df c = df_two_prod(x.hi, y);
    return df_fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
// exact scaling by a power of two
__device__ __forceinline__ Df df_scale(const Df& x, float p2) { return Df(__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)); }
__device__ __forceinline__ Df df_div(const Df& x, const Df& y)
{
    const float th = __fdividef(x.hi, y.hi);
    const Df r = df_mul(y, th);
    // x - y th: the heads cancel exactly (Sterbenz), the rest is the residual
    const float d = __fadd_rn(__fsub_rn(x.hi, r.hi), __fsub_rn(x.lo, r.lo));
    return df_fast_two_sum(th, __fdividef(d, y.hi));
}

__device__ __forceinline__ Df operator-(const Df& x) { return Df(-x.hi, -x.lo); }
__device__ __forceinline__ Df operator+(const Df& x, const Df& y) { return df_add(x, y); }
__device__ __forceinline__ Df operator-(const Df& x, const Df& y) { return df_add(x, -y); }
__device__ __forceinline__ Df operator*(const Df& x, const Df& y) { return df_mul(x, y); }
__device__ __forceinline__ Df operator/(const Df& x, const Df& y) { return df_div(x, y); }
// a double operand: constants fold to two floats; one whose tail is zero takes the
// cheaper float forms
__device__ __forceinline__ Df operator+(const Df& x, double y)
{
    const Df b(y);
    return b.lo == 0.0f ? df_add(x, b.hi) : df_add(x, b);
}
__device__ __forceinline__ Df operator+(double y, const Df& x) { return x + y; }
__device__ __forceinline__ Df operator-(const Df& x, double y) { return x + (-y); }
__device__ __forceinline__ Df operator-(double y, const Df& x) { return (-x) + y; }
__device__ __forceinline__ Df operator*(const Df& x, double y)
{
    const Df b(y);
    return b.lo == 0.0f ? df_mul(x, b.hi) : df_mul(x, b);
}
__device__ __forceinline__ Df operator*(double y, const Df& x) { return x * y; }
__device__ __forceinline__ Df operator/(const Df& x, double y) { return df_div(x, Df(y)); }
__device__ __forceinline__ Df operator/(double y, const Df& x) { return df_div(Df(y), x); }

__device__ __forceinline__ bool operator<(const Df& a, const Df& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(const Df& a, const Df& b) { return b < a; }
__device__ __forceinline__ bool operator<=(const Df& a, const Df& b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(const Df& a, const Df& b) { return !(a < b); }
__device__ __forceinline__ bool operator<(const Df& a, double b) { return a < Df(b); }
__device__ __forceinline__ bool operator>(const Df& a, double b) { return Df(b) < a; }
__device__ __forceinline__ bool operator<=(const Df& a, double b) { return !(Df(b) < a); }
__device__ __forceinline__ bool operator>=(const Df& a, double b) { return !(a < Df(b)); }

// value part (the kinematics templates take a scalar's value for their decisions)
__device__ __forceinline__ Df val(const Df& x) { return x; }
__device__ __forceinline__ Df fabs(const Df& x) { return x.hi < 0.0f ? -x : x; }
// floor as an int (|x| < 2^31)
__device__ __forceinline__ int df_floor(const Df& x)
{
    const float f = floorf(x.hi);
    return (int)f - ((f == x.hi && x.lo < 0.0f) ? 1 : 0);
}

// ------------------------------------------------------------------ elementary functions

// square root: one Newton correction of the correctly rounded float root
__device__ __forceinline__ Df sqrt(const Df& x)
{
    if (!(x.hi > 0.0f)) return Df(x.hi == 0.0f ? 0.0f : __fsqrt_rn(x.hi), 0.0f);
    const float s = __fsqrt_rn(x.hi);
    const Df p = df_two_prod(s, s);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    return df_fast_two_sum(s, __fdividef(d, __fadd_rn(s, s)));
}

// exp(x) for |x| < 87 (0 below, +inf above)
__device__ __forceinline__ Df exp(const Df& x)
{
    if (x.hi > 88.0f) return Df(__int_as_float(0x7f800000), 0.0f);
    if (x.hi < -87.0f) return Df(0.0f, 0.0f);
    // x = k ln 2 + r, |r| <= ln 2 / 2: the 16-bit head of ln 2 times |k| < 2^8 is exact
    const float k = rintf(__fmul_rn(x.hi, 1.44269502162933349609375f));
    constexpr float LN2_HEAD = 0.693145751953125f;
    constexpr Df LN2_TAIL(0.693147180559945309417232121458 - 0.693145751953125);
    Df r = df_add(x, __fmul_rn(-k, LN2_HEAD));
    r = df_add(r, -df_mul(LN2_TAIL, k));
    // s = r / 32; expm1(s) = s + s^2 (1/2 + s (1/6 + s (1/24 + s (1/120 + s / 720)))) with the
    // terms from s^4 on in float (they are below 6e-8 s); omitted: s^7 / 5040 < 4e-18
    const Df s = df_scale(r, 0.03125f);
    const float h = __fmaf_rn(s.hi, __fmaf_rn(s.hi, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f);
    constexpr Df C6(1.0 / 6.0);
    const Df q = df_add(df_mul(s, h), C6);
    const Df p = df_add(df_mul(s, q), 0.5f);
    Df e = df_add(df_mul(df_mul(s, s), p), s);
    // expm1(2a) = expm1(a) (2 + expm1(a)), five times
#pragma unroll
    for (int i = 0; i < 5; ++i) e = df_mul(e, df_add(e, 2.0f));
    const Df y = df_add(e, 1.0f);
    return df_scale(y, __int_as_float(((int)k + 127) << 23));
}

// natural logarithm (NaN below 0, -inf at 0)
__device__ __forceinline__ Df log(const Df& x)
{
    if (!(x.hi > 0.0f)) return Df(x.hi == 0.0f ? __int_as_float(0xff800000) : __int_as_float(0x7fffffff), 0.0f);
    // x = m 2^k, m in [sqrt(1/2), sqrt(2))
    int k;
    float mh = frexpf(x.hi, &k);
    if (mh < 0.70710678118654752f) { mh = __fmul_rn(mh, 2.0f); --k; }
    const Df m(mh, ldexpf(x.lo, -k));
    // y0 = log m to float accuracy; one Newton step on exp(y) = m: y = y0 + m exp(-y0) - 1
    const float y0 = logf(mh);
    const Df c = df_add(df_mul(m, exp(Df(-y0, 0.0f))), -1.0f);
    const Df y = df_add(c, y0);
    constexpr Df LN2(0.693147180559945309417232121458);
    return df_add(y, df_mul(LN2, (float)k));
}

// sin(pi a) and cos(pi a)
__device__ __forceinline__ void sincospi(const Df& a, Df* sp, Df* cp)
{
    // a = n / 2 + r, |r| <= 1/4; t = pi r
    const float n = rintf(__fmul_rn(a.hi, 2.0f));
    const Df r = df_add(a, __fmul_rn(n, -0.5f));
    constexpr Df PI(3.14159265358979323846264338328);
    const Df t = df_mul(r, PI);
    const Df z = df_mul(t, t);   // <= 0.617
    // sin t = t (1 - z/3! + z^2/5! - z^3/7! + z^4/9! - z^5 (1/11! - z/13! + z^2/15!)), the bracket
    // of the last term in float (it is below 2.3e-9); omitted: z^8/17! < 6e-17
    const float fs = __fmaf_rn(z.hi, __fmaf_rn(z.hi, -1.0f / 1307674368000.0f, 1.0f / 6227020800.0f), -1.0f / 39916800.0f);
    constexpr Df S9(1.0 / 362880.0), S7(-1.0 / 5040.0), S5(1.0 / 120.0), S3(-1.0 / 6.0);
    Df ps = df_add(df_mul(z, fs), S9);
    ps = df_add(df_mul(z, ps), S7);
    ps = df_add(df_mul(z, ps), S5);
    ps = df_add(df_mul(z, ps), S3);
    ps = df_add(df_mul(z, ps), 1.0f);
    const Df st = df_mul(t, ps);
    // cos t = 1 - z/2! + z^2/4! - z^3/6! + z^4/8! - z^5/10! + z^6 (1/12! - z/14! + z^2/16!), the
    // bracket in float (below 1.2e-10); omitted: z^9/18! < 3e-18
    const float fc = __fmaf_rn(z.hi, __fmaf_rn(z.hi, 1.0f / 20922789888000.0f, -1.0f / 87178291200.0f), 1.0f / 479001600.0f);
    constexpr Df C10(-1.0 / 3628800.0), C8(1.0 / 40320.0), C6(-1.0 / 720.0), C4(1.0 / 24.0);
    Df pc = df_add(df_mul(z, fc), C10);
    pc = df_add(df_mul(z, pc), C8);
    pc = df_add(df_mul(z, pc), C6);
    pc = df_add(df_mul(z, pc), C4);
    pc = df_add(df_mul(z, pc), -0.5f);
    const Df ct = df_add(df_mul(z, pc), 1.0f);
    const int q = ((int)n) & 3;
    const Df s0 = (q & 1) ? ct : st, c0 = (q & 1) ? st : ct;
    *sp = (q & 2) ? -s0 : s0;
    *cp = (q == 1 || q == 2) ? -c0 : c0;
}

#endif  // __CUDACC__

}  // namespace mf
