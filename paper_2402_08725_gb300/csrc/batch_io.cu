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

// What the per-problem calls apply to one element of kind KIND (0 data, 1 noise, 2 PSFs):
// the value itself with the finiteness check, or w = 1/sigma^2 (sigma = +inf gives 0; NaN or
// sigma <= 0 raises the flag and gives 0).
template <int KIND>
__device__ __forceinline__ float bio_value(float v, bool &bad) {
    if (KIND == 1) {
        if (isinf(v) && v > 0.f) return 0.f;
        if (!(v > 0.f) || isnan(v)) {
            bad = true;
            return 0.f;
        }
        return 1.f / (v * v);
    }
    if (!isfinite(v)) bad = true;
    return v;
}

template <int KIND>
__device__ __forceinline__ float *bio_dst(const BioEntry &b) {
    return KIND == 0 ? b.d : KIND == 1 ? b.w : b.s;
}

constexpr int kBioThreads = 256, kBioPerThread = 8;
constexpr long long kBioChunk = (long long)kBioThreads * kBioPerThread;  // elements (or float4) per block

// Block-contiguous chunks of the packed array; the entry of a chunk's first element is found once
// per thread (binary search), later elements advance from it (entries hold at least one image, far
// more than a chunk's stride).  VEC: every entry's offset and the total are multiples of 4, so each
// float4 of the packed array lies in one entry.
template <int KIND, bool VEC>
__global__ void __launch_bounds__(kBioThreads) bio_copy_kernel(const BioEntry *__restrict__ tab,
                                                               const long long *__restrict__ off, int n,
                                                               const float *__restrict__ src, long long total) {
    const long long units = VEC ? total / 4 : total;
    for (long long c0 = blockIdx.x * kBioChunk; c0 < units; c0 += (long long)gridDim.x * kBioChunk) {
        const long long first = c0 + threadIdx.x;
        if (first >= units) continue;
        int e = entry_of(off, n, VEC ? 4 * first : first);
        long long end = off[e + 1];
        bool bad = false;
        const long long stop = min(units, c0 + kBioChunk);
        for (long long u = first; u < stop; u += kBioThreads) {
            const long long i = VEC ? 4 * u : u;
            while (i >= end) {
                if (bad) atomicOr(tab[e].flag, 1);
                bad = false;
                ++e;
                end = off[e + 1];
            }
            float *dst = bio_dst<KIND>(tab[e]) + (i - off[e]);
            if (VEC) {
                const float4 v = reinterpret_cast<const float4 *>(src)[u];
                float4 r;
                r.x = bio_value<KIND>(v.x, bad);
                r.y = bio_value<KIND>(v.y, bad);
                r.z = bio_value<KIND>(v.z, bad);
                r.w = bio_value<KIND>(v.w, bad);
                *reinterpret_cast<float4 *>(dst) = r;
            } else {
                *dst = bio_value<KIND>(src[u], bad);
            }
        }
        if (bad) atomicOr(tab[e].flag, 1);
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

template <int KIND>
void launch_bio_copy(const BioEntry *tab, const long long *off, int n, const float *src, long long total, bool vec,
                     cudaStream_t st) {
    const long long units = vec ? total / 4 : total;
    long long g = (units + kBioChunk - 1) / kBioChunk;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    if (vec) bio_copy_kernel<KIND, true><<<(int)g, kBioThreads, 0, st>>>(tab, off, n, src, total);
    else bio_copy_kernel<KIND, false><<<(int)g, kBioThreads, 0, st>>>(tab, off, n, src, total);
}

// page-locked host memory <-> device through its mapped address: copies in a kernel, so that they
// take no place in the copy engines' queues
__global__ void hio_copy_kernel(const float *__restrict__ src, float *__restrict__ dst, long long n, bool vec,
                                const double *__restrict__ tsrc, double *__restrict__ tdst) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (tid == 0 && tdst) *tdst = *tsrc;
    if (vec) {
        const long long n4 = n / 4;
        for (long long i = tid; i < n4; i += nt)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(src)[i];
        for (long long i = 4 * n4 + tid; i < n; i += nt) dst[i] = src[i];
    } else {
        for (long long i = tid; i < n; i += nt) dst[i] = src[i];
    }
}

}  // namespace

void launch_bio_flags(const BioEntry *tab, int n, int *out, cudaStream_t st) {
    bio_flags_kernel<<<(n + 255) / 256, 256, 0, st>>>(tab, n, out);
}

void launch_bio_data(const BioEntry *tab, const long long *off, int n, const float *src, long long total, bool vec,
                     cudaStream_t st) {
    launch_bio_copy<0>(tab, off, n, src, total, vec, st);
}

void launch_bio_noise(const BioEntry *tab, const long long *off, int n, const float *src, long long total, bool vec,
                      cudaStream_t st) {
    launch_bio_copy<1>(tab, off, n, src, total, vec, st);
}

void launch_bio_psfs(const BioEntry *tab, const long long *off_s, const long long *off_k, int n, const float *src,
                     long long total_s, long long total_k, bool vec, cudaStream_t st) {
    launch_bio_copy<2>(tab, off_s, n, src, total_s, vec, st);
    bio_kappa_kernel<<<grid_of(total_k), 256, 0, st>>>(tab, off_k, n, total_k);
}

void launch_host_copy(const float *src, float *dst, long long n, const double *tsrc, double *tdst, cudaStream_t st) {
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    long long g = ((vec ? n / 4 : n) + 255) / 256;
    if (g > 152LL * 8) g = 152LL * 8;
    if (g < 1) g = 1;
    hio_copy_kernel<<<(int)g, 256, 0, st>>>(src, dst, n, vec, tsrc, tdst);
}

}  // namespace sr
