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

// TwoSum: s + e = a + b exactly (componentwise).  Every difference is formed
// as an FMA with multiplier -1 (RN(x - y) = fma(-1, y, x)), so that no
// separate negation is issued; the roundings are those of Knuth's sequence.
__device__ __forceinline__ void df_two_sum(float2 a, float2 b, float2& s, float2& e) {
    const float2 m1 = make_float2(-1.f, -1.f);
    s = __fadd2_rn(a, b);
    const float2 nbv = __ffma2_rn(m1, s, a);   // -(s - a)
    const float2 av = __fadd2_rn(s, nbv);      // s - (s - a)
    const float2 da = __ffma2_rn(m1, av, a);   // a - av
    const float2 db = __fadd2_rn(b, nbv);      // b - (s - a)
    e = __fadd2_rn(da, db);
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
// by TwoSum, the low parts and both error terms accumulate in acc.lo.  The
// error terms are carried negated (ne = -e, exact under round-to-nearest)
// so that every step is one paired multiply or FMA.
__device__ __forceinline__ void df_mac(DFPair& acc, float a1, float a2, const DFPair& b) {
    const float2 A1 = make_float2(a1, a1), NA1 = make_float2(-a1, -a1);
    const float2 NA2 = make_float2(-a2, -a2), m1 = make_float2(-1.f, -1.f);
    const float2 p = __fmul2_rn(A1, b.hi);
    float2 ne = __ffma2_rn(NA1, b.hi, p);  // -(a1 b.hi - p)
    ne = __ffma2_rn(NA1, b.lo, ne);
    ne = __ffma2_rn(NA2, b.hi, ne);
    float2 s, err;
    df_two_sum(acc.hi, p, s, err);
    acc.hi = s;
    acc.lo = __fadd2_rn(acc.lo, __ffma2_rn(m1, ne, err));  // acc.lo + (err + e)
}

// acc += sc * b for a scale sc whose components are powers of two (or +-1),
// so that sc * b.hi and sc * b.lo are exact: TwoSum of the high parts with
// the product formed inside the FMAs, 8 paired instructions.
__device__ __forceinline__ void df_add_scaled(DFPair& acc, float2 sc, const DFPair& b) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __ffma2_rn(sc, b.hi, acc.hi);
    const float2 nbv = __ffma2_rn(m1, s, acc.hi);  // -(s - acc.hi)
    const float2 av = __fadd2_rn(s, nbv);
    const float2 da = __ffma2_rn(m1, av, acc.hi);
    const float2 db = __ffma2_rn(sc, b.hi, nbv);   // sc b.hi - (s - acc.hi)
    acc.hi = s;
    acc.lo = __fadd2_rn(__ffma2_rn(sc, b.lo, acc.lo), __fadd2_rn(da, db));
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
