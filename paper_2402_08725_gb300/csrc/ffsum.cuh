// Compensated FP32 sums for the loss reductions.
//
// GB300 executes FP64 at a small fraction of its FP32 rate (two FP64 operations per clock per
// SM), so a per-pixel or per-row FP64 accumulation occupies the FP64 pipe for tens of cycles per
// warp instruction.  The loss sums are carried instead as an unevaluated pair hi + lo of floats:
// each addition records its rounding error exactly (Knuth's TwoSum, The Art of Computer
// Programming vol. 2, sec. 4.2.2) and the pair is renormalised (Dekker's Fast2Sum, 1971), which
// keeps about 2 x 24 significand bits, and each reduced value is widened to double once.  The
// order of the additions is fixed, so the sums stay deterministic.  The code must be compiled
// without reassociation of floating-point additions (nvcc never reassociates them).
#pragma once

namespace sr {

struct FSum {
    float hi, lo;
};

__device__ __forceinline__ FSum fsum_zero() { return {0.f, 0.f}; }

__device__ __forceinline__ FSum fsum_add(FSum a, FSum b) {
    const float s = a.hi + b.hi;
    if (!isfinite(s)) return {s, 0.f};  // an infinite or NaN sum stays what plain addition gives
    const float bv = s - a.hi;
    const float e = ((a.hi - (s - bv)) + (b.hi - bv)) + (a.lo + b.lo);
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ FSum fsum_add(FSum a, float b) { return fsum_add(a, FSum{b, 0.f}); }

// sum over the warp onto lane 0 (a fixed shuffle tree)
__device__ __forceinline__ FSum fsum_warp(FSum v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const FSum w{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = fsum_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double fsum_value(FSum v) { return (double)v.hi + (double)v.lo; }

}  // namespace sr
