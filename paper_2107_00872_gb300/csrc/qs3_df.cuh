// qs3_df.cuh -- double-float arithmetic on the fp32 units: a value is
// hi + lo (two floats, ~48 significant bits).  Products of two floats are
// exact as p + e with e = fma(a, b, -p) (TwoProduct), sums use the
// error-free two-sum (Knuth's TwoSum).  Used by the Gram-Schmidt kernels and
// by the double-float H Phi; GB300 runs fp64 at a small fraction of its
// fp32 rate, so these keep fp64-class accuracy at fp32 throughput.
//
// The products p and the sums that the error terms are formed from use
// __fmul_rn / __fadd_rn / __fsub_rn, which the compiler never contracts
// into a fused multiply-add: a contracted a + x*y would no longer be the
// rounded sum that the two-sum's error term assumes.
#pragma once

#include <cuda_runtime.h>

namespace qs3 {

struct dfl { float hi, lo; };

// s + t = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ float two_sum(float a, float b, float &t) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
__device__ __forceinline__ dfl df_add(dfl a, float b) {     // (a.hi + a.lo) + b
    float e;
    const float s = two_sum(a.hi, b, e);
    const float lo = __fadd_rn(e, a.lo);
    const float hi = __fadd_rn(s, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
// a += x * y (float * float, exact product)
__device__ __forceinline__ dfl df_fma(dfl a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    dfl r = df_add(a, p);
    r.lo += e;
    return r;
}
// a += x * (y.hi + y.lo)  (float times double-float)
__device__ __forceinline__ dfl df_fma2(dfl a, float x, float yh, float yl) {
    const float p = __fmul_rn(x, yh);
    const float e = fmaf(x, yh, -p) + x * yl;
    dfl r = df_add(a, p);
    r.lo += e;
    return r;
}
__device__ __forceinline__ double df_d(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ float2 split_d(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ float4 split2(double2 v) {
    const float2 a = split_d(v.x), b = split_d(v.y);
    return make_float4(a.x, a.y, b.x, b.y);
}

// acc += (ah + al)(bh + bl), dropping al*bl (2^-48 relative); acc is left
// unnormalised (|lo| grows by at most a few ulp of hi per call)
__device__ __forceinline__ void df_mac(dfl &acc, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float t;
    acc.hi = two_sum(acc.hi, p, t);
    acc.lo += t + e;
}
__device__ __forceinline__ dfl df_norm(dfl a) {
    const float s = __fadd_rn(a.hi, a.lo);
    return {s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}
// (a.hi + a.lo)(b.hi + b.lo), renormalised, dropping a.lo * b.lo
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm({p, e});
}
__device__ __forceinline__ dfl df_sum(dfl a, dfl b) {
    float t;
    const float s = two_sum(a.hi, b.hi, t);
    return df_norm({s, t + a.lo + b.lo});
}
__device__ __forceinline__ dfl warp_sum_df(dfl a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        dfl b;
        b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a = df_sum(a, b);
    }
    return a;
}

}  // namespace qs3
