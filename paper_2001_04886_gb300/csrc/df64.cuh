// Double-float ("df64") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// which carries a 48-bit significand. The building blocks are the error-free
// transformations of the published literature: TwoSum (Knuth, TAOCP vol. 2,
// 4.2.2), Fast2Sum (Dekker 1971, valid for |a| >= |b|) and the FMA-based TwoProd
// (p = a*b, e = fma(a, b, -p) is the exact rounding error of the product).
// Every step uses the explicit round-to-nearest intrinsics so that the compiler
// cannot contract or reassociate them (contraction would break exactness).
//
// GB300 issues FP32 FMAs at ~74x its FP64 FMA rate, so a df64 product-accumulate
// (about 12 FP32 instructions) is ~6x faster than a native FP64 one.
#pragma once

#include <cuda_runtime.h>

namespace sstep {

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_norm(float hi, float lo) {
    df64 r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

// x rounded to the nearest df64 (two FP64 -> FP32 conversions and one FP64 subtraction).
__device__ __forceinline__ df64 df_from_double(double x) {
    df64 r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// a + b ("sloppy" addition: error about 2^-48 max(|a|, |b|)).
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

// a * b
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

// a * b + c
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, e));
    return df_norm(s, t);
}

// Dot-product accumulator: the exact product a*b (df64 x df64 or float x float) is
// added with TwoSum into hi; every rounding error collects in lo. lo is folded back
// into hi by normalize() every few terms so that it stays within a few ulps of hi.
struct DfAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(df64 a, df64 b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        float s, t;
        two_sum(hi, p, s, t);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float s, t;
        two_sum(hi, p, s, t);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ void normalize() {
        float s, e;
        fast_two_sum(hi, lo, s, e);
        hi = s;
        lo = e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace sstep
