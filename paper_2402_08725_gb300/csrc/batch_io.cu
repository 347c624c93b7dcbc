// Batched input set-up (sr_batch_set_data / _noise / _psfs): the inputs of every problem of a
// batch, packed in batch order, in one launch per step instead of one call per problem.
//
// Each problem's block sits at its prefix offset in the packed array; a thread finds the problem
// of its element by binary search over the offsets and applies exactly what the per-problem calls
// apply: the data copied with the finiteness check, the noise turned into weights w = 1/sigma^2
// (sigma = +inf gives 0; NaN or sigma <= 0 raises the flag), the PSFs copied with the check and
// folded by D (kappa_fold, the function of the per-problem fold).  Flags are the problems' own.
#include "fold.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

// index of the entry whose [off[e], off[e+1]) holds idx (off[0] = 0, off[n] = total)
__device__ __forceinline__ int entry_of(const long long *__restrict__ off, int n, long long idx) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void bio_data_kernel(const BioEntry *__restrict__ tab, const long long *__restrict__ off, int n,
                                const float *__restrict__ src, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = entry_of(off, n, i);
        const float v = src[i];
        tab[e].d[i - off[e]] = v;
        if (!isfinite(v)) atomicOr(tab[e].flag, 1);
    }
}

__global__ void bio_noise_kernel(const BioEntry *__restrict__ tab, const long long *__restrict__ off, int n,
                                 const float *__restrict__ src, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = entry_of(off, n, i);
        const float s = src[i];
        float wv = 0.f;
        if (isinf(s) && s > 0.f) {
            wv = 0.f;
        } else if (!(s > 0.f) || isnan(s)) {
            atomicOr(tab[e].flag, 1);
        } else {
            wv = 1.f / (s * s);
        }
        tab[e].w[i - off[e]] = wv;
    }
}

__global__ void bio_psf_copy_kernel(const BioEntry *__restrict__ tab, const long long *__restrict__ off, int n,
                                    const float *__restrict__ src, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = entry_of(off, n, i);
        const float v = src[i];
        tab[e].s[i - off[e]] = v;
        if (!isfinite(v)) atomicOr(tab[e].flag, 1);
    }
}

// kappa of every problem from its raw PSFs (already copied): element i of the packed [E][f*f][Tk][Tk]
__global__ void bio_kappa_kernel(const BioEntry *__restrict__ tab, const long long *__restrict__ off, int n,
                                 long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = entry_of(off, n, i);
        const BioEntry &b = tab[e];
        const long long local = i - off[e], per = (long long)b.f * b.f * b.Tk * b.Tk;
        const long long ep = local / per;
        b.kappa[local] = kappa_fold(b.s + ep * b.K * b.K, b.K, b.f, b.Tk, b.tau_lo, local - ep * per);
    }
}

// every entry's input flag into out[] (then cleared): one read-back for the whole batch
__global__ void bio_flags_kernel(const BioEntry *__restrict__ tab, int n, int *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[i] = *tab[i].flag;
        *tab[i].flag = 0;
    }
}

int grid_of(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

void launch_bio_flags(const BioEntry *tab, int n, int *out, cudaStream_t st) {
    bio_flags_kernel<<<(n + 255) / 256, 256, 0, st>>>(tab, n, out);
}

void launch_bio_data(const BioEntry *tab, const long long *off, int n, const float *src, long long total,
                     cudaStream_t st) {
    bio_data_kernel<<<grid_of(total), 256, 0, st>>>(tab, off, n, src, total);
}

void launch_bio_noise(const BioEntry *tab, const long long *off, int n, const float *src, long long total,
                      cudaStream_t st) {
    bio_noise_kernel<<<grid_of(total), 256, 0, st>>>(tab, off, n, src, total);
}

void launch_bio_psfs(const BioEntry *tab, const long long *off_s, const long long *off_k, int n, const float *src,
                     long long total_s, long long total_k, cudaStream_t st) {
    bio_psf_copy_kernel<<<grid_of(total_s), 256, 0, st>>>(tab, off_s, n, src, total_s);
    bio_kappa_kernel<<<grid_of(total_k), 256, 0, st>>>(tab, off_k, n, total_k);
}

}  // namespace sr
