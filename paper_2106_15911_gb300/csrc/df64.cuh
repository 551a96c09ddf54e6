// df64.cuh -- FP64-accurate arithmetic on the FP32 pipe ("double-FP32"): a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// GB300 issues FP32 FMAs about 70 times faster than FP64 ones, so the FMM passes of the FP64 mode
// (S2M, M2M, M2L, L2L, L2T) run in this format.  The operations are the classical error-free
// transformations: Knuth's two-sum and Dekker's fast two-sum for addition, and the exact product
// error of an FMA, a*b - rn(a*b) = fma(a, b, -rn(a*b)), for multiplication (as in the double-double
// arithmetic of Dekker 1971 and Hida, Li, Bailey 2001, here with FP32 components).  Additions are
// the "sloppy" variant (the low parts are added without their own error term): relative error
// about 2^-44 in the worst case of cancellation, 2^-48 otherwise.  All FP32 steps use the _rn
// intrinsics so the compiler cannot contract or reorder them.
#pragma once

#include <cuda_runtime.h>

namespace pfmm {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(int z) : hi((float)z), lo(0.f) {}
    __device__ explicit df64(double d)
    {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
};

__device__ __forceinline__ df64 df_make(float hi, float lo)
{
    df64 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// s + e = a + b exactly, |e| <= ulp(s) / 2 (requires |a| >= |b| or a = 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// s + e = a + b exactly (any order of magnitude)
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

__device__ __forceinline__ df64 operator+(df64 x, df64 y)
{
    float s, e;
    df_two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    return df_fast_two_sum(s, e);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df_make(-x.hi, -x.lo); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64 &operator+=(df64 &x, df64 y)
{
    x = x + y;
    return x;
}

// acc += a * b with one normalisation
__device__ __forceinline__ void mac(df64 &acc, df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, e2;
    df_two_sum(acc.hi, p, s, e2);
    e2 = __fadd_rn(e2, __fadd_rn(e, acc.lo));
    acc = df_fast_two_sum(s, e2);
}
__device__ __forceinline__ void mac(float &acc, float a, float b) { acc += a * b; }
__device__ __forceinline__ void mac(double &acc, double a, double b) { acc += a * b; }

// conversions at the FP64 boundaries of the passes
template <typename R>
__device__ __forceinline__ R from_double(double d)
{
    return R(d);
}
template <>
__device__ __forceinline__ df64 from_double<df64>(double d)
{
    return df64(d);
}
__device__ __forceinline__ double as_double(float x) { return (double)x; }
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(df64 x) { return (double)x.hi + (double)x.lo; }

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void lds4(const df64 *p, df64 (&w)[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 2);
    w[0] = df_make(a.x, a.y);
    w[1] = df_make(a.z, a.w);
    w[2] = df_make(b.x, b.y);
    w[3] = df_make(b.z, b.w);
}

// storage tag of an arithmetic mode: 0 FP64, 1 FP32, 2 double-FP32
template <typename F>
void dispatch_prec(int prec, F &&f)
{
    if (prec == 1) f(float{});
    else if (prec == 2) f(df64{});
    else f(double{});
}

}  // namespace pfmm
