// Float-float accumulation shared by the gather kernels (uniform and batched): a row of products is
// summed as an unevaluated pair of FP32 values, and the rows of a destination are summed as a second
// pair; the destination's value is formed in FP64 once, at the end.
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

// (A, B) += (s, c): a row's pair added into the running pair of a destination.  TwoSum of the leading
// parts, the trailing parts added to its error, then a Fast2Sum renormalisation, so that (A, B) keeps
// about 48 bits of the running total (a double-float sum) without any FP64 instruction: on GB300 the
// FP64 pipe runs at 1/73 of the FP32 rate, and two conversions and two FP64 adds per row and destination
// cost more than the row's 2R+1 FP32 product-sums.
__device__ __forceinline__ void ff_add(float& A, float& B, float s, float c) {
    const float t = __fadd_rn(A, s);
    const float bp = __fsub_rn(t, A);
    const float e = __fadd_rn(__fsub_rn(A, __fsub_rn(t, bp)), __fsub_rn(s, bp));
    const float f = __fadd_rn(e, __fadd_rn(B, c));
    A = __fadd_rn(t, f);
    B = __fsub_rn(f, __fsub_rn(A, t));
}

}  // namespace fdirw
