// df64.cuh -- double-float arithmetic for FP32 pipes (FP64 runs at 1/64 of the FP32 rate on this
// GPU): a value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about
// 48 significant bits.  The error-free transformations are Knuth's TwoSum (TAOCP vol. 2, 4.2.2),
// Dekker's Fast2Sum (1971) and the FMA form of Dekker's product; every operation uses the _rn
// intrinsics, which the compiler never contracts into FMAs.
#pragma once

namespace dvgo {

struct Df {
    float hi, lo;
};

__device__ __forceinline__ Df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ Df df_fast_two_sum(float a, float b) {   // |a| >= |b| (or a == 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ Df df_add(Df a, Df b) {
    Df s = df_two_sum(a.hi, b.hi);
    const Df t = df_two_sum(a.lo, b.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ Df df_neg(Df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ Df df_mul(Df a, Df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return df_fast_two_sum(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi))));
}

__device__ __forceinline__ Df df_mul_f(Df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.hi, b, -p);
    return df_fast_two_sum(p, __fadd_rn(e, __fmul_rn(a.lo, b)));
}

// a / n for a positive integer n < 2^24: the remainder of the rounded quotient is exact in one FMA.
__device__ __forceinline__ Df df_div_n(Df a, float n) {
    const float q1 = __fdiv_rn(a.hi, n);
    const float r = __fmaf_rn(-q1, n, a.hi);
    return df_fast_two_sum(q1, __fdiv_rn(__fadd_rn(r, a.lo), n));
}

__device__ __forceinline__ Df df_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(__dsub_rn(x, (double)hi))};
}

__device__ __forceinline__ bool df_le(Df a, Df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

}  // namespace dvgo
