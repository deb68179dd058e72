// dw.cuh -- double-word (float + float) arithmetic for the CG residual recurrence and
// its inner products.  A value is hi + lo with |lo| <= ulp(hi) / 2, a 48-bit
// significand, computed on the FP32 pipes (the FP64 rate of this part is a small
// fraction of its FP32 rate).  Building blocks: Knuth's TwoSum and the FMA-exact
// product error (Dekker 1971; Joldes, Muller & Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", 2017:
// DWPlusFP and DWTimesFP).  The _rn intrinsics keep the compiler from contracting or
// reordering the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace firm {

// s + e = a + b exactly
__device__ __forceinline__ float2 dw_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

// acc + (ph + pl), ph + pl a double-word (DWPlusDW in its cheap form: the low parts
// are added in one rounding, then renormalised with TwoSum)
__device__ __forceinline__ float2 dw_add(float2 acc, float ph, float pl) {
    const float2 s = dw_two_sum(acc.x, ph);
    return dw_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(acc.y, pl)));
}

// acc += a * b for floats a, b (the product is exact as ph + pe)
__device__ __forceinline__ float2 dw_acc_prod(float2 acc, float a, float b) {
    const float ph = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -ph);
    return dw_add(acc, ph, pe);
}

// acc += r * z for a double-word r and a float z (DWTimesFP)
__device__ __forceinline__ float2 dw_acc_mul(float2 acc, float2 r, float z) {
    const float ph = __fmul_rn(r.x, z);
    const float pe = __fmaf_rn(r.x, z, -ph);
    const float pl = __fmaf_rn(r.y, z, pe);
    return dw_add(acc, ph, pl);
}

// acc += r^2 for a double-word r (r.x^2 + 2 r.x r.y; r.y^2 is below the precision)
__device__ __forceinline__ float2 dw_acc_sq(float2 acc, float2 r) {
    const float ph = __fmul_rn(r.x, r.x);
    const float pe = __fmaf_rn(r.x, r.x, -ph);
    const float pl = __fmaf_rn(__fmul_rn(2.0f, r.x), r.y, pe);
    return dw_add(acc, ph, pl);
}

// r - a * q for a double-word r, a double-word scalar a and a float q
__device__ __forceinline__ float2 dw_sub_mul(float2 r, float2 a, float q) {
    const float ph = __fmul_rn(a.x, q);
    const float pe = __fmaf_rn(a.x, q, -ph);
    const float pl = __fmaf_rn(a.y, q, pe);           // a q = ph + pl
    const float2 s = dw_two_sum(r.x, -ph);
    return dw_two_sum(s.x, __fadd_rn(s.y, __fsub_rn(r.y, pl)));
}

// double -> double-word (host or device; once per scalar)
__host__ __device__ __forceinline__ float2 dw_from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ double dw_to_double(float2 v) { return (double)v.x + (double)v.y; }

// Sum over the 32 lanes of a warp, in double-word; the result is valid in lane 0.
__device__ __forceinline__ float2 dw_warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_down_sync(0xffffffffu, v.x, o);
        const float l = __shfl_down_sync(0xffffffffu, v.y, o);
        v = dw_add(v, h, l);
    }
    return v;
}

}  // namespace firm
