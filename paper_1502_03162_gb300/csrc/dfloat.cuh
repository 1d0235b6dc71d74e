// dfloat.cuh -- double-float ("float-float") arithmetic for sums that must be more accurate
// than FP32 without using FP64: a value is the unevaluated sum hi + lo of two floats.
//
// Built from the error-free transformations of Knuth (TAOCP vol. 2, 4.2.2: TwoSum, the exact
// rounding error of a sum) and Dekker (1971, "A floating-point technique for extending the
// available precision": the exact rounding error of a product, here obtained with one FMA).
// Every operation uses the explicitly rounded intrinsics, so the compiler cannot contract or
// reassociate them.  Relative accuracy of a double-float sum of n terms: about n * 2^-46.
#pragma once

#include <cuda_runtime.h>

namespace hrir {

struct dfl {
    float hi, lo;
};

// s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl df_make(float x) { return {x, 0.f}; }

__device__ __forceinline__ float df_value(dfl a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return {s, e};
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

// acc + a * b, the product's rounding error carried exactly
__device__ __forceinline__ dfl df_fma(dfl acc, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(acc.hi, p, s, e);
    e = __fadd_rn(e, __fadd_rn(acc.lo, pe));
    fast_two_sum(s, e, s, e);
    return {s, e};
}

// acc + a * b with a double-float factor a
__device__ __forceinline__ dfl df_fma_df(dfl acc, dfl a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    const float pe = fmaf(a.hi, b, -p);
    float s, e;
    two_sum(acc.hi, p, s, e);
    e = __fadd_rn(e, __fadd_rn(acc.lo, fmaf(a.lo, b, pe)));
    fast_two_sum(s, e, s, e);
    return {s, e};
}

// sum over the 32 lanes of a warp in a fixed butterfly order (every lane gets the result)
__device__ __forceinline__ dfl df_warp_sum(dfl v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfl w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        // the same operands in the same order on both lanes of a pair: identical results
        v = (threadIdx.x & o) ? df_add(w, v) : df_add(v, w);
    }
    return v;
}

}  // namespace hrir
