// Double-float ("pair of FP32") arithmetic on GB300's paired FP32 pipe.
//
// A double-float number is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2 after normalisation: 48 significand bits, unit roundoff
// ~ 2^-48.  The building blocks are the classical error-free transformations:
// Knuth's TwoSum (a + b = s + e exactly, six additions) and the FMA-based
// TwoProduct (a * b = p + e exactly, e = fma(a, b, -p)).  Every helper works
// on a PAIR of double-float numbers at once (float2 of high parts, float2 of
// low parts) so that each step is one f32x2 instruction (__fadd2_rn,
// __fmul2_rn, __ffma2_rn): the pair is (re, im) of one complex entry or two
// adjacent real entries.  The _rn intrinsics are never contracted or
// reassociated by the compiler, which the transformations rely on.
#pragma once

#include <cuda_runtime.h>

namespace chebfd {

struct DFPair {
    float2 hi, lo;  // component k = hi.k + lo.k
};

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// TwoSum: s + e = a + b exactly (componentwise).
__device__ __forceinline__ void df_two_sum(float2 a, float2 b, float2& s, float2& e) {
    s = __fadd2_rn(a, b);
    const float2 bv = __fadd2_rn(s, df_neg(a));
    const float2 av = __fadd2_rn(s, df_neg(bv));
    e = __fadd2_rn(__fadd2_rn(a, df_neg(av)), __fadd2_rn(b, df_neg(bv)));
}

// Renormalise an accumulated pair (hi may be smaller than lo after cancellation).
__device__ __forceinline__ DFPair df_norm(const DFPair& x) {
    DFPair r;
    df_two_sum(x.hi, x.lo, r.hi, r.lo);
    return r;
}

// acc += a * b for a double-float scalar a = a1 + a2 and a pair b: the exact
// product of the high parts plus the cross terms a1*b.lo + a2*b.hi (the
// a2*b.lo term is below the format's precision); the high parts are added
// by TwoSum, the low parts and both error terms accumulate in acc.lo.
__device__ __forceinline__ void df_mac(DFPair& acc, float a1, float a2, const DFPair& b) {
    const float2 A1 = make_float2(a1, a1), A2 = make_float2(a2, a2);
    const float2 p = __fmul2_rn(A1, b.hi);
    float2 e = __ffma2_rn(A1, b.hi, df_neg(p));
    e = __ffma2_rn(A1, b.lo, e);
    e = __ffma2_rn(A2, b.hi, e);
    float2 s, err;
    df_two_sum(acc.hi, p, s, err);
    acc.hi = s;
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(err, e));
}

// acc += b (pair).
__device__ __forceinline__ void df_add(DFPair& acc, const DFPair& b) {
    float2 s, err;
    df_two_sum(acc.hi, b.hi, s, err);
    acc.hi = s;
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(err, b.lo));
}

// Split a double into hi + lo floats (exact to 2^-48 relative).
__device__ __forceinline__ void df_split(double d, float& hi, float& lo) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}

}  // namespace chebfd
