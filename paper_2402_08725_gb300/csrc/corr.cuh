// Register-blocked 2-D correlation on shared-memory tiles (internal, device code).
#pragma once

#include "common.cuh"

namespace sr {

// Register-blocked 2-D correlation on shared-memory tiles:
//   acc[r] += sum_{jy < Tk} sum_{jx < Tk} Kp[jy][jx] * X[jy][r + jx],   r < R.
// The R-wide input window is a circular register buffer: after the tap jx the slot that
// held X[jx] receives X[jx + R], so each tap costs one shared load of X, a quarter of a
// broadcast float4 load of Kp, and R FMAs.  Each kernel row is summed into its own FP32
// partial before it is added to acc (shorter rounding chains).
// Requirements: kpitch % 4 == 0, Kp 16-byte aligned, Kp[jy][Tk..kpitch) readable, and
// X[jy][0 .. R + Tk - 1] readable.
// ---------------------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void corr_accumulate(float (&acc)[R], const float *__restrict__ X, int xpitch,
                                                const float *__restrict__ Kp, int kpitch, int Tk) {
    const int nfull = Tk / R;
    const int rem = Tk - nfull * R;
    for (int jy = 0; jy < Tk; ++jy) {
        const float *xr = X + jy * xpitch;
        const float *kr = Kp + jy * kpitch;
        float win[R], part[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            win[r] = xr[r];
            part[r] = 0.f;
        }
        int jx0 = 0;
        for (int b = 0; b < nfull; ++b, jx0 += R) {
#pragma unroll
            for (int s4 = 0; s4 < R; s4 += 4) {
                const float4 k4 = *reinterpret_cast<const float4 *>(kr + jx0 + s4);
                const float kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int s = s4 + q;
#pragma unroll
                    for (int r = 0; r < R; ++r) part[r] = fmaf(kk[q], win[(s + r) % R], part[r]);
                    win[s] = xr[jx0 + s + R];
                }
            }
        }
        if (rem) {
#pragma unroll
            for (int s4 = 0; s4 < R; s4 += 4) {
                if (s4 < rem) {
                    const float4 k4 = *reinterpret_cast<const float4 *>(kr + jx0 + s4);
                    const float kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int s = s4 + q;
                        if (s < rem) {
#pragma unroll
                            for (int r = 0; r < R; ++r) part[r] = fmaf(kk[q], win[(s + r) % R], part[r]);
                            win[s] = xr[jx0 + s + R];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += part[r];
    }
}

}  // namespace sr
