// df64.cuh -- double-float arithmetic on the FP32 units: a value is an unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2, 48-bit significand).  Products use the error-free FMA
// transform (p = a*b, e = fma(a, b, -p) is exact) and sums Knuth's TwoSum, i.e. the compensated
// dot product of Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26
// (2005), algorithm Dot2: the result is as accurate as if computed in twice the working precision
// and then rounded.  On GB300 an FP32 FMA issues 58 times as fast as an FP64 one, so the ten FP32
// operations of one double-float multiply-add (df_fma) cost a sixth of a native FP64 FMA.
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

// a += (wh + wl) (xh + xl) in ten FP32 operations.  Knuth's TwoSum of the running sum s and the
// rounded product p = fl(wh xh) gives t = fl(s + p) and the exact residues s - (t - z) and p - z
// (z = t - s); the product's own rounding error wh xh - p is folded into the second residue by one
// FMA, fl(wh xh - z) = fl((p - z) + (wh xh - p)), instead of being formed apart (Dot2 forms it with
// a separate FMA and adds it to the correction).  Both residues and the cross terms wh xl, wl xh
// (relative size 2^-24, rounded once more) go into the correction c.  The error stays of the Dot2
// order (u^2 times the sum of |products| per term, u = 2^-24).  p is formed with __fmul_rn so the
// compiler cannot contract it into the sum s + p (TwoSum needs p as a float).
__device__ __forceinline__ void df_fma(DfAcc& a, float wh, float wl, float xh, float xl)
{
    float p = __fmul_rn(wh, xh);
    float t = a.s + p;
    float z = t - a.s;
    float ar = a.s - (t - z);
    float br = fmaf(wh, xh, -z);
    float c = fmaf(wh, xl, a.c);
    c = fmaf(wl, xh, c);
    a.s = t;
    a.c = c + (ar + br);
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
