// Float-float accumulation shared by the gather kernels (uniform and batched): a row of products is
// summed as an unevaluated pair of FP32 values, then added to an FP64 accumulator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fdirw {

__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

// s + c += q * (hi + lo), all error-free except the q*lo product and the final c update (both ~2^-48
// relative to the running total).  Written with _rn intrinsics so that no step is contracted into an FMA.
__device__ __forceinline__ void ff_madd(float& s, float& c, float q, float2 ch) {
    const float p = __fmul_rn(q, ch.x);
    const float e = __fmaf_rn(q, ch.y, __fmaf_rn(q, ch.x, -p));   // residual of p, plus q*lo
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

}  // namespace fdirw
