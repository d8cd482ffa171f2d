// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA-based TwoProduct.  A complex df value is a float4 (re_hi, re_lo,
// im_hi, im_lo).  Everything here runs on the FP32 pipe.
#pragma once

#include <cuda_runtime.h>

namespace rgf {

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return make_float2(s, e);
}
__device__ __forceinline__ float2 two_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    return make_float2(p, e);
}
// (a.x + a.y) + (b.x + b.y), accurate addition.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    const float2 t = two_sum(a.y, b.y);
    s.y += t.x;
    s = fast_two_sum(s.x, s.y);
    s.y += t.y;
    return fast_two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    float2 p = two_prod(a.x, b.x);
    p.y = fmaf(a.x, b.y, p.y);
    p.y = fmaf(a.y, b.x, p.y);
    return fast_two_sum(p.x, p.y);
}

// Complex df helpers on float4 (re_hi, re_lo, im_hi, im_lo).
__device__ __forceinline__ float2 re_of(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_of(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cdf(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float4 cdf_add(float4 a, float4 b) {
    return cdf(df_add(re_of(a), re_of(b)), df_add(im_of(a), im_of(b)));
}
__device__ __forceinline__ float4 cdf_sub(float4 a, float4 b) {
    return cdf(df_sub(re_of(a), re_of(b)), df_sub(im_of(a), im_of(b)));
}
__device__ __forceinline__ float4 cdf_mul(float4 a, float4 b) {
    const float2 ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
    return cdf(df_sub(df_mul(ar, br), df_mul(ai, bi)), df_add(df_mul(ar, bi), df_mul(ai, br)));
}
// Round a double to the nearest df pair (used once per input block).
__device__ __forceinline__ float2 df_from_double(double x) {
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    return make_float2(hi, lo);
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

}  // namespace rgf
