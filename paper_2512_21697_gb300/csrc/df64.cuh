// df64.cuh -- double-float arithmetic on the FP32 units: a value is an unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2, 48-bit significand).  Products use the error-free FMA
// transform (p = a*b, e = fma(a, b, -p) is exact) and sums Knuth's TwoSum, i.e. the compensated
// dot product of Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26
// (2005), algorithm Dot2: the result is as accurate as if computed in twice the working precision
// and then rounded.  On GB300 an FP32 FMA issues 58 times as fast as an FP64 one, so the dozen
// FP32 operations of one double-float multiply-add cost a fifth of a native FP64 FMA.
#pragma once
#include <cuda_runtime.h>

namespace dg {

// split a double into hi + lo floats
__device__ __forceinline__ float2 df_split(double v)
{
    float h = (float)v;
    float l = (float)(v - (double)h);
    return make_float2(h, l);
}

// running compensated sum: s (the float sum of the rounded products) and c (all rounding errors)
struct DfAcc {
    float s, c;
};

__device__ __forceinline__ void df_zero(DfAcc& a) { a.s = 0.f; a.c = 0.f; }

// a += (wh + wl) (xh + xl): the exact product wh xh as p + e, the two cross terms (whose own
// rounding is 2^-48 relative) into the correction, and p added to s by TwoSum.
__device__ __forceinline__ void df_fma(DfAcc& a, float wh, float wl, float xh, float xl)
{
    float p = wh * xh;
    float e = fmaf(wh, xh, -p);
    e = fmaf(wh, xl, e);
    e = fmaf(wl, xh, e);
    float t = a.s + p;
    float z = t - a.s;
    float err = (a.s - (t - z)) + (p - z);
    a.s = t;
    a.c += err + e;
}

// a = (wh + wl) (xh + xl): the first product of a sum (TwoSum with an empty accumulator returns
// the product itself)
__device__ __forceinline__ void df_mul(DfAcc& a, float wh, float wl, float xh, float xl)
{
    float p = wh * xh;
    float e = fmaf(wh, xh, -p);
    e = fmaf(wh, xl, e);
    a.s = p;
    a.c = fmaf(wl, xh, e);
}

// add another accumulator (sign +1 or -1)
__device__ __forceinline__ void df_add(DfAcc& a, const DfAcc& b, float sign)
{
    float p = sign * b.s;
    float t = a.s + p;
    float z = t - a.s;
    float err = (a.s - (t - z)) + (p - z);
    a.s = t;
    a.c += err + sign * b.c;
}

__device__ __forceinline__ double df_value(const DfAcc& a) { return (double)a.s + (double)a.c; }

}  // namespace dg
