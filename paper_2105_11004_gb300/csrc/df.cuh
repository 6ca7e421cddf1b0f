// Double-float arithmetic shared by the pivoted Cholesky (gramqr.cu) and the triangular solve of
// the right factor (qr.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lev {

// ---- double-float arithmetic: a value is an FP32 pair (hi, lo), |lo| <= ulp(hi) / 2, about 48
// significant bits, operated on with error-free transformations (TwoSum, FMA-based TwoProduct). FP64
// runs at 1/64 of the FP32 rate on GB300, and the Schur updates of the pivoted Cholesky are
// FP64-issue-bound at d = 1,024 in FP64.
__device__ __forceinline__ float2 df_from_double(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }
// a b (TwoProduct of the high parts, cross terms by FMA, renormalised)
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float h = __fadd_rn(p, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// x - a b (TwoSum of the high parts; the low parts and the product's error into the error term)
__device__ __forceinline__ float2 df_sub_mul(float2 x, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -p);
    pe = __fmaf_rn(a.x, b.y, pe);
    pe = __fmaf_rn(a.y, b.x, pe);
    const float s = __fsub_rn(x.x, p);
    const float bb = __fsub_rn(s, x.x);
    float err = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    err = __fadd_rn(err, __fsub_rn(x.y, pe));
    const float h = __fadd_rn(s, err);
    return make_float2(h, __fsub_rn(err, __fsub_rn(h, s)));
}
// 1 / sqrt(v) for a positive double-float v: an FP32 estimate, one FP32 Newton step, then one step
// y + y (1 - v y^2) / 2 with the residual formed in double-float (to about 2^-46)
__device__ __forceinline__ float2 df_inv_sqrt(float2 v) {
    float y = rsqrtf(v.x);
    y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f, v.x), __fmul_rn(y, y), 1.5f));
    const float yy = __fmul_rn(y, y);
    const float yye = __fmaf_rn(y, y, -yy);
    const float2 t = df_mul(v, make_float2(yy, yye));
    const float res = __fadd_rn(__fsub_rn(1.0f, t.x), -t.y);
    const float corr = __fmul_rn(__fmul_rn(0.5f, y), res);
    const float h = __fadd_rn(y, corr);
    return make_float2(h, __fsub_rn(corr, __fsub_rn(h, y)));
}
// order-preserving keys of an FP32 value and of a double-float (hi first, then lo); 0 marks "none"
__device__ __forceinline__ unsigned order_key32(float v) {
    const unsigned b = __float_as_uint(v);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long df_key(float2 v) {
    return ((unsigned long long)order_key32(v.x) << 32) | order_key32(v.y);
}
__device__ __forceinline__ unsigned long long df_bits(float2 v) {
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 df_of_bits(unsigned long long b) {
    return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}

}  // namespace lev
