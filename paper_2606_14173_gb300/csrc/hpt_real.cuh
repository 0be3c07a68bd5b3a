// Arithmetic of the coherent chain: native FP64 or double-float ("df64": the unevaluated sum
// hi + lo of two floats, ~48-bit significand).
//
// The double-float operations follow the error-free transformations of Dekker (1971) and
// Knuth (TAOCP vol. 2): TwoSum for exact sums, and TwoProd through a fused multiply-add for
// exact products; renormalisation by QuickTwoSum.  Only additions, subtractions and
// explicit __fmaf_rn / __fmul_rn appear in the transformations, so the compiler's FMA
// contraction cannot change them.
#pragma once
#include <cuda_runtime.h>
#include "hpt_internal.h"

namespace hpt {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df mkdf(float h, float l) { df r; r.hi = h; r.lo = l; return r; }

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return mkdf(s, e);
}

__device__ __forceinline__ df quick_two_sum(float a, float b)   // requires |a| >= |b|
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return mkdf(s, e);
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return mkdf(p, e);
}

__device__ __forceinline__ df operator+(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df operator-(df a) { return mkdf(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df mul_f(df a, float b)
{
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df add_f(df a, float b)
{
    df s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return quick_two_sum(s.hi, s.lo);
}

// quotient from three partial digits with a float reciprocal of the divisor's head
__device__ __forceinline__ df operator/(df a, df b)
{
    float inv = __frcp_rn(b.hi);
    float q1 = __fmul_rn(a.hi, inv);
    df r = a - mul_f(b, q1);
    float q2 = __fmul_rn(r.hi, inv);
    r = r - mul_f(b, q2);
    float q3 = __fmul_rn(r.hi, inv);
    return add_f(quick_two_sum(q1, q2), q3);
}

// square root: float root, then one correction from the exact residual a - x^2
__device__ __forceinline__ df df_sqrt(df a)
{
    if (!(a.hi > 0.0f)) return mkdf(0.0f, 0.0f);
    float x = __fsqrt_rn(a.hi);
    df r = a - two_prod(x, x);
    float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, x));
    return quick_two_sum(x, c);
}

// ---------------------------------------------------------------- generic Real interface
template <class R> struct RealOps;

template <> struct RealOps<double> {
    static __device__ __forceinline__ double rc(const RC &c) { return c.d; }
    static __device__ __forceinline__ double f(float x) { return (double)x; }
    static __device__ __forceinline__ double fromd(double x) { return x; }
    static __device__ __forceinline__ double to_d(double x) { return x; }
    static __device__ __forceinline__ float to_f(double x) { return (float)x; }
    static __device__ __forceinline__ double mulf(double a, float b) { return a * (double)b; }
    static __device__ __forceinline__ double addf(double a, float b) { return a + (double)b; }
    static __device__ __forceinline__ double sqrt_(double a) { return a > 0.0 ? sqrt(a) : 0.0; }
    static __device__ __forceinline__ int floor_i(double a) { return (int)floor(a); }
    static __device__ __forceinline__ float frac_f(double a) { return (float)(a - floor(a)); }
    static __device__ __forceinline__ double load(const double *p64, const float2 *pdf, int i)
    {
        (void)pdf;
        return __ldg(p64 + i);
    }
    // cos and sin of 2 pi u for a 24-bit fraction u
    static __device__ __forceinline__ void sincos2pi(float u, const float4 *, double &s, double &c)
    {
        sincospi(2.0 * (double)u, &s, &c);
    }
};

template <> struct RealOps<df> {
    static __device__ __forceinline__ df rc(const RC &c) { return mkdf(c.hi, c.lo); }
    static __device__ __forceinline__ df f(float x) { return mkdf(x, 0.0f); }
    static __device__ __forceinline__ df fromd(double x)
    {
        float h = __double2float_rn(x);
        return mkdf(h, __double2float_rn(x - (double)h));
    }
    static __device__ __forceinline__ double to_d(df x) { return (double)x.hi + (double)x.lo; }
    static __device__ __forceinline__ float to_f(df x) { return __fadd_rn(x.hi, x.lo); }
    static __device__ __forceinline__ df mulf(df a, float b) { return mul_f(a, b); }
    static __device__ __forceinline__ df addf(df a, float b) { return add_f(a, b); }
    static __device__ __forceinline__ df sqrt_(df a) { return df_sqrt(a); }
    static __device__ __forceinline__ int floor_i(df a)
    {
        float fl = floorf(a.hi);
        if (fl == a.hi && a.lo < 0.0f) fl -= 1.0f;
        return (int)fl;
    }
    static __device__ __forceinline__ float frac_f(df a)
    {
        float f = __fsub_rn(a.hi, floorf(a.hi));   // exact
        f = __fadd_rn(f, a.lo);
        return __fsub_rn(f, floorf(f));
    }
    static __device__ __forceinline__ df load(const double *p64, const float2 *pdf, int i)
    {
        (void)p64;
        float2 v = __ldg(pdf + i);
        return mkdf(v.x, v.y);
    }
    // cos/sin(2 pi u), u = k/256 + b with b < 2^-8: table value of the head times the
    // Taylor series of the tail x = 2 pi b, |x| < 0.0246.  The leading terms x^2/2 and x^3/6
    // are formed in double-float (a float would leave absolute errors of ~1e-11 in cos);
    // the remaining terms are below 1.5e-8 and 7.5e-11, so float keeps their error under
    // 1e-15, and the truncation after x^7 leaves less than 1e-17.
    static __device__ __forceinline__ void sincos2pi(float u, const float4 *tab, df &s, df &c)
    {
        unsigned q = (unsigned)(u * 16777216.0f);       // exact: u has 24 fractional bits
        unsigned k = q >> 16;
        float b = (float)(q & 0xFFFFu) * (1.0f / 16777216.0f);
        const df two_pi = mkdf(6.28318548202514648f, -1.74845553e-07f);
        const df sixth = mkdf(0.166666672f, -4.96705388e-09f);
        df x = mul_f(two_pi, b);
        df x2 = x * x;
        df x3 = x2 * x;
        float x2f = x2.hi;
        float ct = x2f * x2f * (1.0f / 24.0f) * (1.0f - x2f * (1.0f / 30.0f));   // x^4/24 - x^6/720
        float st = x3.hi * x2f * (1.0f / 120.0f) * (1.0f - x2f * (1.0f / 42.0f)); // x^5/120 - x^7/5040
        df cb = add_f(mkdf(1.0f, 0.0f) - mul_f(x2, 0.5f), ct);
        df sb = add_f(x - x3 * sixth, st);
        float4 t = __ldg(tab + k);                       // (cos.hi, cos.lo, sin.hi, sin.lo)
        df ca = mkdf(t.x, t.y), sa = mkdf(t.z, t.w);
        c = ca * cb - sa * sb;
        s = sa * cb + ca * sb;
    }
};

}  // namespace hpt
