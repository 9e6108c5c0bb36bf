// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits, on the
// FP32 pipe (B300's FP64 rate is ~1/70 of its FP32 rate, and a conversion
// between the two formats costs as much as an FP64 operation, so values
// enter and leave this form once per vertex or tet, not per operation).
// Error-free transformations: the two-sum of Knuth (TAOCP vol. 2,
// sec. 4.2.2), the fast two-sum of Dekker (1971, |a| >= |b|), and the exact
// product by fused multiply-add.  Addition is Dekker's add2 (the high parts
// by two-sum, the low parts added to its error): its error is bounded by
// ~2^-46 (|a| + |b|) rather than by the result, which for the elastic
// terms (displacements u = x - X, small next to x) stays below the FP64
// path's own rounding of x - X.
#pragma once
#include <cuda_runtime.h>

namespace gmcp {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_make(float a) { return {a, 0.f}; }
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_fast_two_sum(p, e);
}
// a b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) { return df_add(df_mul(a, b), c); }
// a b - c d
__device__ __forceinline__ dfl df_mms(dfl a, dfl b, dfl c, dfl d) { return df_sub(df_mul(a, b), df_mul(c, d)); }
// a / b by two steps of long division (quotient digit, exact remainder)
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float q1 = a.hi / b.hi;
    const dfl r = df_sub(a, df_mulf(b, q1));
    const float q2 = r.hi / b.hi;
    const dfl r2 = df_sub(r, df_mulf(b, q2));
    const float q3 = r2.hi / b.hi;
    const dfl q = df_fast_two_sum(q1, q2);
    return df_add(q, df_make(q3));
}
// hi + lo rounded to FP64 / an FP64 value split into the pair
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl df_from_double(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
// a > b for pairs in the normal form (hi the rounded value of the sum)
__device__ __forceinline__ bool df_gt(dfl a, float b) { return a.hi > b || (a.hi == b && a.lo > 0.f); }

}  // namespace gmcp
