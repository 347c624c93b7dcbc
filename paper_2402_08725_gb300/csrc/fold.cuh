// The D-folded narrow-PSF kernels (internal; shared by the per-problem and the batched set-up).
#pragma once

namespace sr {

// kappa_{i,phi}(tau) for tau in [tau_lo, tau_lo + Tk)^2, element idx of [f*f][Tk][Tk] of one epoch
// (phi = phy*f + phx): kappa(t) = sum_{a,b<f} s[t + (a,b) + o] with t = f*tau - phi, o = K/2, the
// sum over the f x f block of D taken in FP64 in a fixed order.
__device__ __forceinline__ float kappa_fold(const float *__restrict__ si, int K, int f, int Tk, int tau_lo,
                                            long long idx) {
    long long r = idx;
    const int tx = (int)(r % Tk);
    r /= Tk;
    const int ty = (int)(r % Tk);
    r /= Tk;
    const int ph = (int)r;
    const int phy = ph / f, phx = ph - phy * f, o = K / 2;
    const int t_y = f * (tau_lo + ty) - phy;
    const int t_x = f * (tau_lo + tx) - phx;
    double acc = 0.0;
    for (int a = 0; a < f; ++a) {
        const int qy = t_y + a + o;
        if (qy < 0 || qy >= K) continue;
        for (int b = 0; b < f; ++b) {
            const int qx = t_x + b + o;
            if (qx < 0 || qx >= K) continue;
            acc += (double)si[qy * K + qx];
        }
    }
    return (float)acc;
}

}  // namespace sr
