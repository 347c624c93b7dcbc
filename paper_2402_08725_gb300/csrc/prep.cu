// Input preparation: inverse-variance weights and finiteness checks (sm_103a).
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sr {

// w = 1/sigma^2 (diagonal C of Eq. 4 / Eq. 10); sigma = +inf gives w = 0 (masked pixel).
// sigma that is NaN or <= 0 raises the flag.
__global__ void inv_var_kernel(const float *sigma, float *w, long long n, int *bad) {  // in place: w may alias sigma
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float s = sigma[i];
        float wv = 0.f;
        if (isinf(s) && s > 0.f) {
            wv = 0.f;
        } else if (!(s > 0.f) || isnan(s)) {
            atomicOr(bad, 1);
        } else {
            wv = 1.f / (s * s);
        }
        w[i] = wv;
    }
}

__global__ void check_finite_kernel(const float *__restrict__ x, long long n, int *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!isfinite(x[i])) atomicOr(bad, 1);
    }
}

__global__ void flag_to_nan_kernel(const int *flag, double *loss) {
    if (*flag) *loss = __longlong_as_double(0x7ff8000000000000LL);
}

static int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return g < 1 ? 1 : (int)g;
}

void launch_inv_var(const float *sigma, float *w, long long n, int *bad_flag, cudaStream_t st) {
    inv_var_kernel<<<grid_for(n), 256, 0, st>>>(sigma, w, n, bad_flag);
}

void launch_check_finite(const float *x, long long n, int *bad_flag, cudaStream_t st) {
    check_finite_kernel<<<grid_for(n), 256, 0, st>>>(x, n, bad_flag);
}

void launch_flag_to_nan(const int *flag, double *loss, cudaStream_t st) { flag_to_nan_kernel<<<1, 1, 0, st>>>(flag, loss); }

}  // namespace sr
