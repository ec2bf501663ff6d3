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
// 1 / a, a != 0 (normal): q, the hardware's approximate 1 / a.hi
// (rcp.approx, about 23 bits), refined by one FP32 Newton step, then one
// Newton step whose residual 1 - a q is formed in double-float (A. H. Karp
// and P. Markstein, "High-precision division and square root", ACM TOMS 23
// (1997) 561-589).  In an emulation against a float64 reference its
// relative error stays at 1.35e-14 over 1e-3 .. 1e3, the same as with the
// IEEE reciprocal as the first approximation.
__device__ __forceinline__ float df_rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ dfloat df_rcp(dfloat a) {
    float q = df_rcp_approx(a.hi);
    q = __fmaf_rn(q, __fmaf_rn(-a.hi, q, 1.0f), q);
    const dfloat r = df_sub(df_from(1.0f), df_mul_f(a, q));  // 1 - a q
    return df_fast_two_sum(q, __fmul_rn(r.hi, q));
}

// The per-stage phase-change source of Eq. 24, C1 a + C2 sqrt(a) with
// a = t + ts (t the FP32 stage temperature, ts, C1, C2 in double-float),
// rounded once to FP32 at the end.  sqrt(a): y, the hardware's approximate
// 1 / sqrt(a.hi) (rsqrt.approx, about 22 bits), refined by one FP32 Newton
// step for the reciprocal root; s0 = a.hi y; then one Newton step for the
// root whose residual a - s0^2 is formed with a fused multiply-add (Karp and
// Markstein, as above): about 45 bits (checked against a float64 reference
// in an emulation: within 0.66 FP32 ulp of the result even where the two
// products cancel to 1e-6 of their size, against 0.59 with a correctly
// rounded FP32 root and an exact 1 / (2 s0) as the first approximation).
// The two products are summed with an error-free sum of their high parts.
__device__ __forceinline__ float df_rsqrt_approx(float x) {  // x > 0, normal
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float df_source(dfloat c1, dfloat c2, float t, dfloat ts) {
    dfloat a = df_two_sum(t, ts.hi);
    a = df_fast_two_sum(a.hi, __fadd_rn(a.lo, ts.lo));
    float y = df_rsqrt_approx(a.hi);
    y = __fmaf_rn(__fmul_rn(0.5f, y), __fmaf_rn(-__fmul_rn(a.hi, y), y, 1.0f), y);
    const float s0 = __fmul_rn(a.hi, y);
    const float e = __fadd_rn(__fmaf_rn(-s0, s0, a.hi), a.lo);  // a - s0^2
    const dfloat s = df_fast_two_sum(s0, __fmul_rn(__fmul_rn(0.5f, y), e));
    const dfloat p1 = df_mul(c1, a), p2 = df_mul(c2, s);
    const dfloat h = df_two_sum(p1.hi, p2.hi);
    return __fadd_rn(h.hi, __fadd_rn(h.lo, __fadd_rn(p1.lo, p2.lo)));
}

}  // namespace lbmgb
