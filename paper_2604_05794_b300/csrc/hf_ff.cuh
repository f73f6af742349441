// hf_ff.cuh - float-float (double-single) arithmetic on FP32 for exact pixel decisions.
#pragma once

#include <cuda_runtime.h>

namespace hf_ff {

// Error-free transformations on FP32 (Knuth two-sum, FMA two-product).  A value is hi + lo with
// |lo| <= ulp(hi)/2; about 44 significant bits survive the operations below, which places a
// projected pixel coordinate within ~1e-10 px of its exact value, so floor() picks the same pixel
// as an exact evaluation except for coordinates within that distance of a pixel edge.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}
// r0 p0 + r1 p1 + r2 p2 + t, all inputs exact FP32
__device__ __forceinline__ ff ff_dot3_plus(float r0, float r1, float r2, float p0, float p1, float p2, float t) {
    ff s = ff_add(two_prod(r0, p0), two_prod(r1, p1));
    s = ff_add(s, two_prod(r2, p2));
    return ff_add(s, ff{t, 0.0f});
}
// x / y
__device__ __forceinline__ ff ff_div(ff x, ff y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    ff p = two_prod(q1, y.hi);
    float r = __fsub_rn(x.hi, p.hi);  // exact (Sterbenz): p.hi is within a factor 2 of x.hi
    r = __fsub_rn(r, p.lo);
    r = __fadd_rn(r, x.lo);
    r = __fmaf_rn(-q1, y.lo, r);
    float q2 = __fdiv_rn(r, y.hi);
    return fast_two_sum(q1, q2);
}
// f * a + c, f and c exact FP32
__device__ __forceinline__ ff ff_affine(float f, ff a, float c) {
    ff m = two_prod(f, a.hi);
    m.lo = __fmaf_rn(f, a.lo, m.lo);
    m = fast_two_sum(m.hi, m.lo);
    return ff_add(m, ff{c, 0.0f});
}
// floor(hi + lo) for a normalised pair
__device__ __forceinline__ float ff_floor(ff x) {
    float f = floorf(x.hi);
    if (f == x.hi && x.lo < 0.0f) f -= 1.0f;
    return f;
}

}  // namespace hf_ff
