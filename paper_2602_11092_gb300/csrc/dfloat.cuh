// Double-float arithmetic on the FP32 pipe: a number is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2, about 44 significant bits.
// Built from error-free transformations: Knuth's two-sum (the exact rounding
// error of a + b), Dekker's fast two-sum for |a| >= |b|, and the exact product
// error a * b - fl(a * b) from one fused multiply-add.  Every step uses the
// round-to-nearest intrinsics, which the compiler never contracts or
// reassociates, so the error terms stay exact.
//
// Used where a sum cancels far below its terms (Glynn's permanent formula) or
// runs over many terms (renormalisation), so that no kernel needs the FP64
// pipe (1/64 of the FP32 rate on this GPU).
#pragma once
#include <cuda_runtime.h>

namespace slos {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_zero() { return {0.f, 0.f}; }

// s + e = a + b exactly
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly
__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ dfl df_add_f(dfl x, float b) {
    const dfl s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const dfl p = two_prod(x.hi, y.hi);
    const float e = __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ float df_float(dfl x) { return __fadd_rn(x.hi, x.lo); }

// complex double-float
struct cdfl {
    dfl re, im;
};

__device__ __forceinline__ cdfl cdf_mul(cdfl a, cdfl b) {
    return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

__device__ __forceinline__ cdfl cdf_add(cdfl a, cdfl b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }

__device__ __forceinline__ cdfl cdf_sub(cdfl a, cdfl b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }

}  // namespace slos
