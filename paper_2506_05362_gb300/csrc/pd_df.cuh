// Double-float arithmetic: a value is held as an unevaluated pair hi + lo of
// FP32 numbers with |lo| <= ulp(hi)/2, giving ~48-bit significands from FP32
// units only.  Error-free transformations after Dekker (1971) and Knuth
// (TAOCP vol. 2, Sec. 4.2.2), in the formulation of Hida, Li and Bailey's
// double-double library, specialised to FP32 and FMA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// The state pairs (u and v of every node) are kept on the FP64 grid: hi + lo is
// exactly a double, and splitting that double again gives the same pair.  A pair
// is then converted to FP64 and back without change, so a state read out and sent
// back is recognised as the live one, and a run restarted from a saved state goes
// on bit for bit as the uninterrupted run.
//
// df_from_double(x): hi = RN(x), lo = x - hi rounded towards zero.  hi + lo is a
// double (lo is either x - hi itself, when that fits 24 bits, or its truncation,
// whose last bit then lies at or above the double grid of x), and |lo| reaches
// ulp(hi)/2 only when x - hi is exactly that tie, which RN resolved to an even
// hi; so RN(hi + lo) = hi and the split of hi + lo is the pair again.
__device__ __forceinline__ df df_from_double(double x)
{
    df r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rz(__dsub_rn(x, (double)r.hi));
    return r;
}

// A normalised pair (RN(hi + lo) = hi, as a two-sum leaves it) moved onto the FP64
// grid: lo replaced by RN64(hi + lo) - hi, which is exact in FP64 and fits FP32, so
// hi + lo becomes exactly the double nearest the old pair (a move of at most 2^-53
// of the value).  It is computed in FP32, without FP64 instructions: the grid of
// hi + lo has spacing q = 2^(e - 52), e the exponent of hi + lo (that of hi, one less
// when hi is a power of two and lo points towards zero); only a lo below 2^23 q in
// size can have bits under q, and for it adding and subtracting M = 2^23 q (with
// lo's sign) rounds it to a multiple of q, nearest and ties to even, as RN64 does
// (hi / q is even).  hi = 0, or a grid finer than FP32's smallest subnormal, leaves
// the pair as it is.
__device__ __forceinline__ df df_on_fp64_grid(df a)
{
    const uint32_t hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
    int eq = (int)((hb >> 23) & 0xffu) - 127 - 52;  // log2 q
    if ((hb & 0x7fffffu) == 0u && ((hb ^ lb) & 0x80000000u) && a.lo != 0.f) eq -= 1;
    if (eq >= -149) {
        const float t = __uint_as_float((uint32_t)(eq + 23 + 127) << 23);  // 2^23 q, a normal FP32
        if (fabsf(a.lo) < t) {
            const float m = __uint_as_float(__float_as_uint(t) | (lb & 0x80000000u));
            a.lo = __fsub_rn(__fadd_rn(a.lo, m), m);
        }
    }
    return a;
}

// the double nearest hi + lo (exact for the state pairs, which lie on the FP64
// grid); every kernel converts with this one formula, so all see the same value
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
