// Double-float arithmetic on pairs of FP32 numbers (value = hi + lo with |lo| at most half
// an ulp of hi), used where the mixed-precision trajectory is kept beyond FP32: Knuth's
// TwoSum (the exact error of a rounded sum, no ordering assumption) and Dekker's Fast2Sum
// (the same when |a| >= |b|). The _rn intrinsics keep the compiler from contracting or
// reassociating the error terms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdmpt {
namespace dd {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (ahi + alo) + (bhi + blo), renormalised into (hi, lo)
__device__ __forceinline__ void add(float ahi, float alo, float bhi, float blo, float& hi,
                                    float& lo) {
    float s, e;
    two_sum(ahi, bhi, s, e);
    e = __fadd_rn(e, __fadd_rn(alo, blo));
    fast_two_sum(s, e, hi, lo);
}

// (ahi + alo) + b for one FP32 b
__device__ __forceinline__ void add1(float ahi, float alo, float b, float& hi, float& lo) {
    float s, e;
    two_sum(ahi, b, s, e);
    e = __fadd_rn(e, alo);
    fast_two_sum(s, e, hi, lo);
}

// TF32 split of an FP32 value for the split-TF32 engine: hi = rna_tf32(v), lo = rna_tf32(v - hi)
__device__ __forceinline__ void tf32_split(float v, float& h, float& l) {
    uint32_t a, b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(a) : "f"(v));
    h = __uint_as_float(a);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(__fsub_rn(v, h)));
    l = __uint_as_float(b);
}

}  // namespace dd
}  // namespace cdmpt
