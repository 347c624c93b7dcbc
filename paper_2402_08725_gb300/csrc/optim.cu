// Fused optimiser update with projection (sm_103a).
//
// The paper minimises its losses with gradient-based optimisers, AdaBelief among them
// (sec. 2.4).  AdaBelief here is the published update of Zhuang et al. (2020):
//     m <- b1 m + (1-b1) g;   s <- b2 s + (1-b2) (g - m)^2 + eps;
//     theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(s / (1 - b2^t)) + eps)
// Adam uses g^2 in place of (g - m)^2 and no eps inside s.  After the update each element is
// clamped to its group's lower bound (a >= 0; PSF alpha and beta bounded away from their poles).
// One element per thread, HBM-bound: reads theta, g, m, v, group id and writes theta, m, v.
// The step counter t lives in device memory so that a captured graph can be replayed.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sr {

__global__ void opt_prologue_kernel(long long *t, float *bc, float beta1, float beta2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const long long tn = *t + 1;
        *t = tn;
        bc[0] = (float)(1.0 - pow((double)beta1, (double)tn));
        bc[1] = (float)(1.0 - pow((double)beta2, (double)tn));
    }
}

__global__ void opt_update_kernel(long long n, float *__restrict__ params, const float *__restrict__ grad,
                                  float *__restrict__ m, float *__restrict__ v, const uint8_t *__restrict__ group,
                                  OptimArgs a, const float *__restrict__ bc) {
    const float bc1 = bc[0], bc2 = bc[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int gr = group[i];
        const float g = grad[i];
        const float mi = a.beta1 * m[i] + (1.f - a.beta1) * g;
        float vi;
        if (a.kind == SR_ADABELIEF) {
            const float dev = g - mi;
            vi = a.beta2 * v[i] + (1.f - a.beta2) * dev * dev + a.eps;
        } else {
            vi = a.beta2 * v[i] + (1.f - a.beta2) * g * g;
        }
        m[i] = mi;
        v[i] = vi;
        const float step = a.lr[gr] * (mi / bc1) / (sqrtf(vi / bc2) + a.eps);
        params[i] = fmaxf(params[i] - step, a.lo[gr]);
    }
}

void launch_opt_step(long long n, float *params, const float *grad, float *m, float *v, const uint8_t *group,
                     const OptimArgs &a, long long *t_dev, float *bc_dev, cudaStream_t st) {
    opt_prologue_kernel<<<1, 32, 0, st>>>(t_dev, bc_dev, a.beta1, a.beta2);
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    opt_update_kernel<<<(int)blocks, 256, 0, st>>>(n, params, grad, m, v, group, a, bc_dev);
}

}  // namespace sr
