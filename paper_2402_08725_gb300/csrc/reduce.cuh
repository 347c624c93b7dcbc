// Deterministic block reductions (internal, device code).
#pragma once

#include "common.cuh"
#include "ffsum.cuh"

namespace sr {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// This thread's share of sum_{s < n} v[s] over the block (slots s = tid + k blockDim): four
// interleaved partial sums (k mod 4), each in increasing s, combined as (p0 + p1) + (p2 + p3), so
// that four loads per thread are in flight; the same result for the same block size.
__device__ __forceinline__ double strided_sum4(const double *__restrict__ v, long long n) {
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    const long long b = blockDim.x;
    long long s = threadIdx.x;
    for (; s + 3 * b < n; s += 4 * b) {
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] += v[s + u * b];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (s + u * b < n) p[u] += v[s + u * b];
    return (p[0] + p[1]) + (p[2] + p[3]);
}

// Deterministic block sum of two doubles (fixed shuffle tree, warps summed in order).
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*red)[kThreads / 32]) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            sa += red[0][i];
            sb += red[1][i];
        }
        a = sa;
        b = sb;
    }
}

// The same over compensated FP32 pairs (FP64 only for the two results, on thread 0).
__device__ __forceinline__ void block_fsum2(FSum a, FSum b, float2 (*red)[kThreads / 32], double &oa, double &ob) {
    a = fsum_warp(a);
    b = fsum_warp(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = make_float2(a.hi, a.lo);
        red[1][wid] = make_float2(b.hi, b.lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FSum sa = fsum_zero(), sb = fsum_zero();
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            sa = fsum_add(sa, FSum{red[0][i].x, red[0][i].y});
            sb = fsum_add(sb, FSum{red[1][i].x, red[1][i].y});
        }
        oa = fsum_value(sa);
        ob = fsum_value(sb);
    }
}

}  // namespace sr
