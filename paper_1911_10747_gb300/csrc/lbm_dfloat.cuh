// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significand bits, computed on
// the FP32 units.  The error-free transformations are Dekker's (T. J. Dekker,
// "A floating-point technique for extending the available precision",
// Numer. Math. 18 (1971) 224-242) and Knuth's two-sum (TAOCP Vol. 2,
// Sec. 4.2.2); products use the fused multiply-add for the exact low part.
// Every sum and product goes through the _rn intrinsics so that the
// compiler cannot contract or reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace lbmgb {

struct dfloat {
    float hi, lo;
};

// a + b = s + e exactly (any magnitudes)
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// a + b = s + e exactly, for |a| >= |b|
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a b = p + e exactly
__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfloat df_from(float a) { return {a, 0.0f}; }
__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ float df_to_float(dfloat a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat s = df_two_sum(a.hi, b.hi);
    const dfloat t = df_two_sum(a.lo, b.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    dfloat p = df_two_prod(a.hi, b.hi);
    const float c = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return df_fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
    dfloat p = df_two_prod(a.hi, b);
    return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// 1 / a and sqrt(a): the FP32 result of the high part refined by one Newton
// step whose residual is formed in double-float (A. H. Karp and P. Markstein,
// "High-precision division and square root", ACM TOMS 23 (1997) 561-589).
// 1 / a, a != 0:
__device__ __forceinline__ dfloat df_rcp(dfloat a) {
    const float q = __frcp_rn(a.hi);
    const dfloat r = df_sub(df_from(1.0f), df_mul_f(a, q));  // 1 - a q
    return df_fast_two_sum(q, __fmul_rn(r.hi, q));
}
// sqrt(a), a > 0:
__device__ __forceinline__ dfloat df_sqrt(dfloat a) {
    const float s = __fsqrt_rn(a.hi);
    const dfloat r = df_sub(a, df_two_prod(s, s));          // a - s^2
    return df_fast_two_sum(s, __fmul_rn(r.hi, __fdiv_rn(0.5f, s)));
}

}  // namespace lbmgb
