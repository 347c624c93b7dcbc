// Noise propagation to the starlet coefficients (sec. 2.3, App. B): the prior weights W by
// Monte Carlo.
//
// Realisation r draws a standard normal field z_r on the fine grid, forms
// (C^)^-1 dd = z_r / sigma_eff^ (the co-added noise map, sigma_eff^-2 = sum_i sigma_i^-2,
// replicated over the f x f fine pixels of each data pixel), applies S_1^T (correlation with
// epoch 1's narrow PSF, the transpose of the zero-padded "same" convolution) and the starlet
// analysis.  W_j is the standard deviation of the detail plane w_{j+1}: per coefficient over
// the realisations (the map), and pooled over the plane's coefficients and the realisations
// (the one number per scale that the prior takes).
//
// Random numbers: normal number n of stream `seed` comes from Philox4x64-10 (Salmon et al.
// 2011) block n/4 with counter (n/4, 0, 0, 0) and key (seed, 0); the block's words (0,1) and
// (2,3) give two Box-Muller pairs from 24-bit uniforms u = ((w >> 40) + 1) 2^-24, cos then sin.
// Realisation r uses the numbers r F^2 .. r F^2 + F^2 - 1 in row-major pixel order.
//
// Work per batch of B realisations (all resident in L2):
//   noise_draw_kernel      x[b]  = z / sigma_eff^                     (one Philox block a thread)
//   noise_corr_kernel      y[b]  = S_1^T x[b]                          (FP32, 2 F^2 K^2 flop each)
//   noise_row_kernel       t[b]  = row pass of level j on c_j[b]
//   noise_col_stats_kernel c_{j+1}[b] = column pass; w = c_j - c_{j+1}; FP64 sum and sum of
//                          squares of w over the batch, in a fixed order, into per-segment
//                          accumulators
// and at the end noise_map_kernel / noise_scale_kernel reduce the segments in a fixed order.
// The correlation dominates: it is bound by FP32 FMA issue.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sr {
namespace {

// ---- counter-based normals ---------------------------------------------------------------

constexpr uint64_t kPhM0 = 0xD2E7470EE14C6C93ULL, kPhM1 = 0xCA5A826395121157ULL;
constexpr uint64_t kPhW0 = 0x9E3779B97F4A7C15ULL, kPhW1 = 0xBB67AE8584CAA73BULL;

__device__ __forceinline__ void philox4x64_10(uint64_t &c0, uint64_t &c1, uint64_t &c2, uint64_t &c3, uint64_t k0,
                                              uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(kPhM0, c0), lo0 = kPhM0 * c0;
        const uint64_t hi1 = __umul64hi(kPhM1, c2), lo1 = kPhM1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += kPhW0;
        k1 += kPhW1;
    }
}

__device__ __forceinline__ float uniform24(uint64_t w) { return (float)((w >> 40) + 1) * 0x1p-24f; }

// x[b][u] = z(seed, (r0 + b) F^2 + u) * isig[u] for the n = B F^2 numbers of the batch.
__global__ void __launch_bounds__(256) noise_draw_kernel(const float *__restrict__ isig, int F, uint64_t seed,
                                                         long long r0, int B, float *__restrict__ x) {
    const long long FF = (long long)F * F;
    const long long n0 = r0 * FF, n1 = n0 + (long long)B * FF;
    const long long blk0 = n0 >> 2, blk1 = (n1 - 1) >> 2;
    for (long long blk = blk0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; blk <= blk1;
         blk += (long long)gridDim.x * blockDim.x) {
        uint64_t c0 = (uint64_t)blk, c1 = 0, c2 = 0, c3 = 0;
        philox4x64_10(c0, c1, c2, c3, seed, 0);
        float z[4];
        {
            const float r = sqrtf(-2.f * logf(uniform24(c0)));
            float s, c;
            sincospif(2.f * uniform24(c1), &s, &c);
            z[0] = r * c;
            z[1] = r * s;
        }
        {
            const float r = sqrtf(-2.f * logf(uniform24(c2)));
            float s, c;
            sincospif(2.f * uniform24(c3), &s, &c);
            z[2] = r * c;
            z[3] = r * s;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long n = 4 * blk + e;
            if (n < n0 || n >= n1) continue;
            const long long u = n % FF;
            x[n - n0] = z[e] * isig[u];
        }
    }
}

// ---- S_1^T: zero-padded correlation, register-blocked ---------------------------------------
//
// y[v] = sum_{qy,qx} s[qy][qx] x[vy + qy - o][vx + qx - o]   (o = K/2; x = 0 outside the grid)
//
// A block of kCorrWarps warps computes a TY x TX tile of one realisation.  Lane l of warp w
// owns output rows w*2*RY + (l/16)*RY + i (i < RY) and the two column groups 4(l%16) + j and
// 64 + 4(l%16) + j (j < 4).  The kernel rows are taken KC at a time (KC >= RY): the x rows the
// chunk needs ((TY + KC - 1) x (TX + KP), zero-filled outside the grid) and the chunk's kernel
// rows (zero beyond K) are staged in shared memory.  For x row r of the thread's window, output
// row i uses kernel row r - i, so rows r < RY - 1 and r >= KC feed only part of the RY outputs:
// corr_row takes the range of i as template arguments and no FMA is spent on a missing row.
// Per group of four kernel columns, two float4 of x (a quarter-warp reads 128 consecutive
// bytes: no bank conflict) and one broadcast float4 of s per output row feed 32 FMAs per row;
// the FMAs are ordered by kernel column so that consecutive ones share their s operand.

constexpr int kCorrRY = 4;
constexpr int kCorrWarps = 4;
constexpr int kCorrTY = 2 * kCorrRY * kCorrWarps;  // 32 output rows per block
constexpr int kCorrTX = 128;                       // 16 column groups x 2 x 4 columns
constexpr int kCorrThreads = 32 * kCorrWarps;
constexpr int kCorrMinBlocks = 3;                  // blocks per SM the chunk size aims for

size_t corr_smem_bytes(int KP, int KC) {
    return sizeof(float) * ((size_t)(kCorrTY + KC - 1) * (kCorrTX + KP) + (size_t)KC * KP);
}

// x row r of the window against kernel rows r - i for i in [ILO, IHI)
template <int ILO, int IHI>
__device__ __forceinline__ void corr_row(float (&acc)[kCorrRY][2][4], const float4 *__restrict__ xp,
                                         const float *__restrict__ ss, int r, int KP) {
    const int G = KP / 4;
    float4 A0 = xp[0], A1 = xp[16];
#pragma unroll 4
    for (int g = 0; g < G; ++g) {
        const float4 B0 = xp[g + 1], B1 = xp[g + 17];
        const float xa[2][8] = {{A0.x, A0.y, A0.z, A0.w, B0.x, B0.y, B0.z, B0.w},
                                {A1.x, A1.y, A1.z, A1.w, B1.x, B1.y, B1.z, B1.w}};
#pragma unroll
        for (int i = ILO; i < IHI; ++i) {
            const float4 sv = reinterpret_cast<const float4 *>(ss + (size_t)(r - i) * KP)[g];
            const float se[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][h][j] = fmaf(se[e], xa[h][j + e], acc[i][h][j]);
        }
        A0 = B0;
        A1 = B1;
    }
}

__global__ void __launch_bounds__(kCorrThreads, kCorrMinBlocks)
    noise_corr_kernel(const float *__restrict__ x, const float *__restrict__ s, int F, int K, int KP, int KC,
                      float *__restrict__ y) {
    static_assert(kCorrRY == 4, "the head and tail rows below are written out for RY = 4");
    extern __shared__ float4 corr_sm4[];
    const int XR = kCorrTY + KC - 1, XW = kCorrTX + KP;
    float *xs = reinterpret_cast<float *>(corr_sm4);
    float *ss = xs + (size_t)XR * XW;
    const int b = blockIdx.z, ty0 = blockIdx.y * kCorrTY, tx0 = blockIdx.x * kCorrTX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, o = K / 2;
    const int row0 = warp * 2 * kCorrRY + (lane >> 4) * kCorrRY, col0 = 4 * (lane & 15);
    const float *xb = x + (size_t)b * F * F;

    float acc[kCorrRY][2][4];
#pragma unroll
    for (int i = 0; i < kCorrRY; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][0][j] = acc[i][1][j] = 0.f;

    for (int q0 = 0; q0 < K; q0 += KC) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < XR * XW; idx += kCorrThreads) {
            const int t = idx / XW, c = idx - t * XW;
            const int gy = ty0 - o + q0 + t, gx = tx0 - o + c;
            xs[idx] = (gy >= 0 && gy < F && gx >= 0 && gx < F) ? xb[(size_t)gy * F + gx] : 0.f;
        }
        for (int idx = threadIdx.x; idx < KC * KP; idx += kCorrThreads) {
            const int qy = idx / KP, qx = idx - qy * KP, q = q0 + qy;
            ss[idx] = (q < K && qx < K) ? s[(size_t)q * K + qx] : 0.f;
        }
        __syncthreads();
        const float *xrow = xs + (size_t)row0 * XW + col0;
        auto xp = [&](int r) { return reinterpret_cast<const float4 *>(xrow + (size_t)r * XW); };
        corr_row<0, 1>(acc, xp(0), ss, 0, KP);
        corr_row<0, 2>(acc, xp(1), ss, 1, KP);
        corr_row<0, 3>(acc, xp(2), ss, 2, KP);
        for (int r = kCorrRY - 1; r < KC; ++r) corr_row<0, kCorrRY>(acc, xp(r), ss, r, KP);
        corr_row<1, 4>(acc, xp(KC), ss, KC, KP);
        corr_row<2, 4>(acc, xp(KC + 1), ss, KC + 1, KP);
        corr_row<3, 4>(acc, xp(KC + 2), ss, KC + 2, KP);
    }
    float *yb = y + (size_t)b * F * F;
#pragma unroll
    for (int i = 0; i < kCorrRY; ++i) {
        const int vy = ty0 + row0 + i;
        if (vy >= F) break;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int vx = tx0 + 64 * h + col0 + j;
                if (vx < F) yb[(size_t)vy * F + vx] = acc[i][h][j];
            }
    }
}

// ---- batched starlet analysis with per-coefficient moments ---------------------------------

constexpr float kH0 = 0.0625f, kH1 = 0.25f, kH2 = 0.375f;  // B3 spline (1,4,6,4,1)/16

__device__ __forceinline__ int reflect(int t, int F) { return t < 0 ? -t : (t > F - 1 ? 2 * (F - 1) - t : t); }

// t[b][y][x] = sum_m h[m] c[b][y][reflect(x + m step)]
__global__ void __launch_bounds__(256) noise_row_kernel(const float *__restrict__ c, float *__restrict__ t, int F,
                                                        int step, long long total) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int xx = (int)(idx % F);
        const float *row = c + (idx - xx);
        t[idx] = kH0 * (row[reflect(xx - 2 * step, F)] + row[reflect(xx + 2 * step, F)]) +
                 kH1 * (row[reflect(xx - step, F)] + row[reflect(xx + step, F)]) + kH2 * row[xx];
    }
}

// Column pass of level j for the realisations of segment blockIdx.y, pixel u per thread:
// c_{j+1} = column filter of t, w = c_j - c_{j+1} (c updated in place: only this thread reads or
// writes c[b][u]); the segment's sums of w and w^2, taken over b in increasing order (groups of
// four in FP32, the groups in FP64), are added to acc1/acc2[seg][j][u].
__global__ void __launch_bounds__(256) noise_col_stats_kernel(float *__restrict__ c, const float *__restrict__ t,
                                                              int F, int step, int B, int S, int J1, int j,
                                                              double *__restrict__ acc1, double *__restrict__ acc2) {
    const long long FF = (long long)F * F;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= FF) return;
    const int seg = blockIdx.y;
    const int b0 = (int)((long long)B * seg / S), b1 = (int)((long long)B * (seg + 1) / S);
    const int yy = (int)(u / F), xx = (int)(u - (long long)yy * F);
    const long long o_m2 = (long long)reflect(yy - 2 * step, F) * F + xx, o_p2 = (long long)reflect(yy + 2 * step, F) * F + xx;
    const long long o_m1 = (long long)reflect(yy - step, F) * F + xx, o_p1 = (long long)reflect(yy + step, F) * F + xx;
    double s1 = 0.0, s2 = 0.0;
    int b = b0;
    for (; b + 4 <= b1; b += 4) {  // four realisations' loads issued before their arithmetic
        float tv[4][5], cv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float *tb = t + (b + k) * FF;
            tv[k][0] = tb[o_m2];
            tv[k][1] = tb[o_m1];
            tv[k][2] = tb[u];
            tv[k][3] = tb[o_p1];
            tv[k][4] = tb[o_p2];
            cv[k] = c[(b + k) * FF + u];
        }
        // the four realisations summed in FP32 (in order), then added to the FP64 sums: a quarter
        // of the FP64 operations, which run at a small fraction of the FP32 rate
        float q1 = 0.f, q2 = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float cn = kH0 * (tv[k][0] + tv[k][4]) + kH1 * (tv[k][1] + tv[k][3]) + kH2 * tv[k][2];
            const float w = cv[k] - cn;
            c[(b + k) * FF + u] = cn;
            q1 += w;
            q2 = fmaf(w, w, q2);
        }
        s1 += (double)q1;
        s2 += (double)q2;
    }
    for (; b < b1; ++b) {
        const float *tb = t + b * FF;
        const float cn = kH0 * (tb[o_m2] + tb[o_p2]) + kH1 * (tb[o_m1] + tb[o_p1]) + kH2 * tb[u];
        float *cb = c + b * FF + u;
        const float w = *cb - cn;
        *cb = cn;
        s1 += (double)w;
        s2 += (double)w * (double)w;
    }
    const long long k = ((long long)seg * J1 + j) * FF + u;
    acc1[k] += s1;
    acc2[k] += s2;
}

// W_map[j][u] = sample std (n - 1) of w_{j+1}[u] over the n realisations (segments summed in order).
__global__ void __launch_bounds__(256) noise_map_kernel(const double *__restrict__ acc1,
                                                        const double *__restrict__ acc2, long long per_seg, int S,
                                                        int n, float *__restrict__ W_map) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= per_seg) return;
    double t1 = 0.0, t2 = 0.0;
    for (int s = 0; s < S; ++s) {
        t1 += acc1[s * per_seg + k];
        t2 += acc2[s * per_seg + k];
    }
    const double mean = t1 / n, var = (t2 - n * mean * mean) / (n - 1);
    W_map[k] = (float)sqrt(var > 0.0 ? var : 0.0);
}

// W_scale[j] = sample std (n F^2 - 1) of every coefficient of plane j: one block per plane, a
// strided per-thread sum then a fixed-shape tree.
constexpr int kScaleThreads = 256;
__global__ void __launch_bounds__(kScaleThreads) noise_scale_kernel(const double *__restrict__ acc1,
                                                                    const double *__restrict__ acc2, long long FF,
                                                                    int J1, int S, int n, float *__restrict__ W) {
    __shared__ double r1[kScaleThreads], r2[kScaleThreads];
    const int j = blockIdx.x;
    const long long per_seg = FF * J1;
    double t1 = 0.0, t2 = 0.0;
    for (long long u = threadIdx.x; u < FF; u += kScaleThreads)
        for (int s = 0; s < S; ++s) {
            t1 += acc1[s * per_seg + j * FF + u];
            t2 += acc2[s * per_seg + j * FF + u];
        }
    r1[threadIdx.x] = t1;
    r2[threadIdx.x] = t2;
    __syncthreads();
    for (int h = kScaleThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            r1[threadIdx.x] += r1[threadIdx.x + h];
            r2[threadIdx.x] += r2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = (double)n * (double)FF, mean = r1[0] / m, var = (r2[0] - m * mean * mean) / (m - 1.0);
        W[j] = (float)sqrt(var > 0.0 ? var : 0.0);
    }
}

// 1/sigma_eff on the fine grid; flags (bit 0) a NaN or non-positive sigma and (bit 1) a
// non-finite PSF value.
__global__ void __launch_bounds__(256) noise_isig_kernel(const float *__restrict__ sigma, const float *__restrict__ s1,
                                                         int N, int f, int E, int K, float *__restrict__ isig,
                                                         int *__restrict__ flag) {
    const int F = f * N;
    const long long FF = (long long)F * F, KK = (long long)K * K;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < FF || u < KK;
         u += (long long)gridDim.x * blockDim.x) {
        if (u < KK && !isfinite(s1[u])) atomicOr(flag, 2);
        if (u >= FF) continue;
        const int yy = (int)(u / F), xx = (int)(u % F);
        const long long p = (long long)(yy / f) * N + xx / f;
        double iv = 0.0;
        for (int i = 0; i < E; ++i) {
            const float sg = sigma[(long long)i * N * N + p];
            if (isnan(sg) || sg <= 0.f) atomicOr(flag, 1);
            else if (isfinite(sg)) iv += 1.0 / ((double)sg * (double)sg);
        }
        isig[u] = (float)sqrt(iv);
    }
}

struct DevBufs {
    std::vector<void *> ptrs;
    ~DevBufs() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T> sr_status alloc(T **p, size_t count) {
        *p = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("sr_noise_weights: cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                      cudaGetErrorString(e));
            return SR_ERR_OOM;
        }
        ptrs.push_back(*p);
        return SR_OK;
    }
};

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" sr_status sr_noise_weights(int N, int f, int K, int J, int E, const float *sigma_dev,
                                      const float *s1_dev, int n_real, uint64_t seed, float *W_host,
                                      float *W_map_dev, sr_noise_timing *timing, void *cuda_stream) {
    if (!sigma_dev || !s1_dev || (!W_host && !W_map_dev)) {
        set_error("sr_noise_weights: sigma, s1 and at least one output are required");
        return SR_ERR_ARG;
    }
    if (N < 1 || f < 1 || K < 1 || E < 1 || J < 2 || n_real < 2 || (long long)f * N > 65535) {
        set_error("sr_noise_weights: need N, f, K, E >= 1, J >= 2, n_real >= 2 and f N <= 65535");
        return SR_ERR_SHAPE;
    }
    const int F = f * N;
    if (J > 31 || 2LL * (1LL << (J - 2)) > F - 1) {
        set_error("sr_noise_weights: the starlet needs 2 * 2^(J-2) <= F - 1 (F = %d, J = %d)", F, J);
        return SR_ERR_SHAPE;
    }
    const int KP = (K + 3) & ~3;
    int dev = 0, sms = 0, optin = 0, per_sm = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SR_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // kernel rows per chunk (at least RY; rows beyond K are zero): the largest that lets
    // kCorrMinBlocks blocks share an SM (1 KB reserved per block), else the largest that fits one
    int KC = 0;
    for (int kc : {64, 32, 16, 8})
        if (kCorrMinBlocks * (corr_smem_bytes(KP, std::max(std::min(kc, K), kCorrRY)) + 1024) <= (size_t)per_sm) {
            KC = std::max(std::min(kc, K), kCorrRY);
            break;
        }
    if (!KC)
        for (int kc : {32, 16, 8})
            if (corr_smem_bytes(KP, std::max(std::min(kc, K), kCorrRY)) <= (size_t)optin) {
                KC = std::max(std::min(kc, K), kCorrRY);
                break;
            }
    if (!KC) {
        set_error("sr_noise_weights: PSF size K = %d needs more shared memory than a block has", K);
        return SR_ERR_UNSUPPORTED;
    }
    const size_t corr_smem = corr_smem_bytes(KP, KC);
    SR_CUDA(cudaFuncSetAttribute(noise_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)corr_smem));
    int occ = 0;
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, noise_corr_kernel, kCorrThreads, corr_smem));
    occ = std::max(occ, 1);

    // batch: whole waves of correlation blocks, two F x F float buffers per realisation within 64 MB
    const long long FF = (long long)F * F;
    const int tiles_x = (F + kCorrTX - 1) / kCorrTX, tiles_y = (F + kCorrTY - 1) / kCorrTY;
    const long long tiles = (long long)tiles_x * tiles_y, resident = (long long)occ * sms;
    const long long bmax = std::max(1LL, (64LL << 20) / (2 * 4 * FF));
    long long B = std::max(1LL, (std::max(1LL, bmax * tiles / resident) * resident) / tiles);
    B = std::min({B, bmax, (long long)n_real, 65535LL});
    // segments of the moment sums: enough threads in the column pass to fill the GPU
    const int S = (int)std::max(1LL, std::min({16LL, B, (sms * 2048LL + FF - 1) / FF}));
    const int J1 = J - 1;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    DevBufs bufs;
    float *isig, *xbuf, *cbuf, *wsc;
    double *acc1, *acc2;
    int *flag;
    sr_status rc;
    if ((rc = bufs.alloc(&isig, FF)) || (rc = bufs.alloc(&xbuf, B * FF)) || (rc = bufs.alloc(&cbuf, B * FF)) ||
        (rc = bufs.alloc(&acc1, (size_t)S * J1 * FF)) || (rc = bufs.alloc(&acc2, (size_t)S * J1 * FF)) ||
        (rc = bufs.alloc(&wsc, J1)) || (rc = bufs.alloc(&flag, 1)))
        return rc;
    SR_CUDA(cudaMemsetAsync(acc1, 0, sizeof(double) * S * J1 * FF, st));
    SR_CUDA(cudaMemsetAsync(acc2, 0, sizeof(double) * S * J1 * FF, st));
    SR_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));

    cudaEvent_t ev[5] = {};
    const bool timed = timing != nullptr;
    double t_draw = 0, t_corr = 0, t_star = 0, t_fin = 0;
    int launches = 0;
    auto destroy_events = [&]() {
        for (cudaEvent_t &e : ev)
            if (e) cudaEventDestroy(e), e = nullptr;
    };
    if (timed)
        for (cudaEvent_t &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                destroy_events();
                return cuda_fail(cudaGetLastError(), "cudaEventCreate");
            }
    auto elapsed = [&](int a, int b) -> double {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return ms;
    };

    const int gs = (int)std::min<long long>((std::max(FF, (long long)K * K) + 255) / 256, sms * 8LL);
    noise_isig_kernel<<<gs, 256, 0, st>>>(sigma_dev, s1_dev, N, f, E, K, isig, flag);
    ++launches;
    for (long long r0 = 0; r0 < n_real; r0 += B) {
        const int Bb = (int)std::min(B, (long long)n_real - r0);
        if (timed) cudaEventRecord(ev[0], st);
        const long long nblk = ((r0 + Bb) * FF - 1) / 4 - (r0 * FF) / 4 + 1;
        noise_draw_kernel<<<(int)std::min<long long>((nblk + 255) / 256, sms * 16LL), 256, 0, st>>>(
            isig, F, seed, r0, Bb, xbuf);
        if (timed) cudaEventRecord(ev[1], st);
        noise_corr_kernel<<<dim3(tiles_x, tiles_y, Bb), kCorrThreads, corr_smem, st>>>(xbuf, s1_dev, F, K, KP, KC,
                                                                                       cbuf);
        if (timed) cudaEventRecord(ev[2], st);
        const long long total = Bb * FF;
        const int Sb = std::min(S, Bb);
        for (int j = 0; j < J1; ++j) {
            noise_row_kernel<<<(int)std::min<long long>((total + 255) / 256, sms * 16LL), 256, 0, st>>>(
                cbuf, xbuf, F, 1 << j, total);
            noise_col_stats_kernel<<<dim3((unsigned)((FF + 255) / 256), Sb), 256, 0, st>>>(
                cbuf, xbuf, F, 1 << j, Bb, Sb, J1, j, acc1, acc2);
        }
        launches += 2 + 2 * J1;
        if (timed) {
            cudaEventRecord(ev[3], st);
            const cudaError_t e = cudaEventSynchronize(ev[3]);
            if (e != cudaSuccess) {
                destroy_events();
                return cuda_fail(e, "noise propagation batch");
            }
            t_draw += elapsed(0, 1);
            t_corr += elapsed(1, 2);
            t_star += elapsed(2, 3);
        }
    }
    if (timed) cudaEventRecord(ev[0], st);
    if (W_map_dev) {
        const long long per = (long long)J1 * FF;
        noise_map_kernel<<<(unsigned)((per + 255) / 256), 256, 0, st>>>(acc1, acc2, per, S, n_real, W_map_dev);
        ++launches;
    }
    noise_scale_kernel<<<J1, kScaleThreads, 0, st>>>(acc1, acc2, FF, J1, S, n_real, wsc);
    ++launches;
    if (timed) cudaEventRecord(ev[4], st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        destroy_events();
        return cuda_fail(e, "noise propagation kernels");
    }
    int hflag = 0;
    e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && W_host) e = cudaMemcpyAsync(W_host, wsc, sizeof(float) * J1, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        destroy_events();
        return cuda_fail(e, "sr_noise_weights");
    }
    if (timed) {
        t_fin = elapsed(0, 4);
        timing->draw_ms = t_draw;
        timing->corr_ms = t_corr;
        timing->starlet_ms = t_star;
        timing->final_ms = t_fin;
        timing->launches = launches;
        timing->batch = (int)B;
        destroy_events();
    }
    if (hflag) {
        set_error("sr_noise_weights: %s", (hflag & 1) ? "sigma holds a NaN or a value <= 0" : "s1 is not finite");
        return SR_ERR_NONFINITE;
    }
    return SR_OK;
}
