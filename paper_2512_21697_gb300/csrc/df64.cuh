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

// split a double into hi + lo floats with integer operations on its bit pattern, no FP64 instruction:
// hi is v truncated to 24 significant bits (sign, exponent rebiased, the top 23 mantissa bits), lo
// the remaining 29 mantissa bits converted once to float (one rounding to 24 bits), so
// |v - (hi + lo)| <= 2^-48 |v| and |lo| < ulp(hi).  |v| < 2^-126 gives (+-0, 0) (the float range's
// underflow); lo is 0 when hi is within 2^52 of the smallest normal float (v below 2^-74);
// infinities and NaN keep their kind in hi.  The FP64 pipe of this part issues a 64th of the FP32
// rate, and a conversion split (df_split) costs it three conversions and a subtraction.
__device__ __forceinline__ float2 df_split_bits(double v)
{
    const unsigned int h = (unsigned int)__double2hiint(v), l = (unsigned int)__double2loint(v);
    const unsigned int sgn = h & 0x80000000u;
    const int E = (int)((h >> 20) & 0x7ffu);
    const int ef = E - 896;   // the float's biased exponent
    if (E == 0x7ff)
        return make_float2(__int_as_float((int)(sgn | 0x7f800000u | (((h & 0xfffffu) | l) ? 0x400000u : 0u))), 0.f);
    if (ef <= 0) return make_float2(__int_as_float((int)sgn), 0.f);
    if (ef >= 255) return make_float2(__int_as_float((int)(sgn | 0x7f800000u)), 0.f);
    const unsigned int hb = sgn | ((unsigned int)ef << 23) | ((h & 0xfffffu) << 3) | (l >> 29);
    float lo = 0.f;
    if (ef > 52) {   // the low 29 bits weigh 2^(ef - 179) each: a normal float scale
        lo = __int2float_rn((int)(l & 0x1fffffffu)) * __int_as_float((ef - 52) << 23);
        if (sgn) lo = -lo;
    }
    return make_float2(__int_as_float((int)hb), lo);
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

// a += (wh + wl) (xh + xl) in six FP32 operations, for an accumulator whose float part a.s holds a
// fixed offset sigma = 1.5 * 2^k plus the running sum of the rounded products, where the caller
// guarantees sum |wh xh| <= 2^(k-2) over everything the accumulator will take.  Then a.s stays in
// [1.25, 1.75] * 2^k, one binade with the fixed unit 2^(k-23): t = fl(a.s + wh xh) (one FMA) and
// d = t - a.s are exact (Sterbenz: both in the binade), and the part of the product that did not
// fit the grid, wh xh - d (|.| <= 2^(k-24)), is formed by a second FMA with one rounding of
// relative size 2^-24.  That residue and the cross terms wh xl, wl xh go into a.c.  This is
// Dekker's Fast2Sum, whose condition |a.s| >= |wh xh| the offset makes hold for every term, with
// the summand taken straight from the FMA (the offset is the error-free extraction idea of Rump,
// Ogita and Oishi, "Accurate floating-point summation part I", SIAM J. Sci. Comput. 31 (2008)).
// The value is (a.s - sigma) + a.c, a.s - sigma exact.  Error for m terms: m 2^-48 2^k from the
// residues plus the roundings of a.c (|a.c| <= m 2^(k-24) + the cross terms), at most about
// 3 m^2 2^-48 2^k: the Dot2 form of df_fma (m^2 u^2 sum |p|, u = 2^-24) with 2^k <= 8 times the
// caller's bound in place of sum |p|, for six operations instead of ten.
__device__ __forceinline__ void df_fma_off(DfAcc& a, float wh, float wl, float xh, float xl)
{
    float t = fmaf(wh, xh, a.s);
    float d = t - a.s;
    float e = fmaf(wh, xh, -d);
    float c = a.c + e;
    c = fmaf(wh, xl, c);
    a.c = fmaf(wl, xh, c);
    a.s = t;
}

// the offset sigma = 1.5 * 2^k of df_fma_off from its biased exponent byte (k + 127)
__device__ __forceinline__ float df_offset(unsigned int eb) { return __int_as_float((int)((eb << 23) | 0x400000u)); }

// biased exponent byte of the offset for a bound B >= sum |wh xh| (B >= 0): the least k with
// 2^(k-2) >= 1.0625 B (the factor covers the bound's own FP32 roundings).  B below 1e-30, zero or
// not a number gives a tiny normal offset (the products are then zero).
__device__ __forceinline__ unsigned int df_offset_byte(float B)
{
    float bm = B * 1.0625f;
    if (!(bm >= 1e-30f)) bm = 1e-30f;
    unsigned int eb = ((unsigned int)__float_as_int(bm) >> 23) & 0xffu;   // bm < 2^(eb - 126)
    return eb + 3u > 254u ? 254u : eb + 3u;
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
