// Double-float arithmetic: a value is held as an unevaluated pair hi + lo of
// FP32 numbers with |lo| <= ulp(hi)/2, giving ~48-bit significands from FP32
// units only.  Error-free transformations after Dekker (1971) and Knuth
// (TAOCP vol. 2, Sec. 4.2.2), in the formulation of Hida, Li and Bailey's
// double-double library, specialised to FP32 and FMA.
#pragma once

#include <cuda_runtime.h>

struct df {
    float hi, lo;
};

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, requires |a| >= |b| or a == 0
__device__ __forceinline__ void quick_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    quick_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    df r;
    quick_two_sum(s, e, r.hi, r.lo);
    return r;
}

// double-float times a float
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    df r;
    quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df r;
    quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_from_double(double x)
{
    df r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

// the double nearest hi + lo (exact whenever lo lies within 29 bits of hi); every
// kernel converts with this one formula, so all see the same FP64 value
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
