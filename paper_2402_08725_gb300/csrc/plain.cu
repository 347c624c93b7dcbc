// The plain per-epoch form of the deconvolution loss and gradient (sm_103a): the literal
// operator order of Eq. 10, one epoch at a time, each step its own launch, intermediates in
// global memory.  It is the measured baseline for the fused, D-folded, batched form.
//
// Per epoch i:  raster  f_i = h + sum_k a_ki r_k            (fine grid)
//               conv    y_i = S_i f_i                      (K x K taps per fine pixel)
//               resid   M_i = D y_i + f^2 Gamma_i, r, chi^2, e = -w r
//               up      D^T e                              (block broadcast)
//               corr    G_i = S_i^T D^T e, and sum_i G_i   (K x K taps per fine pixel)
//               psgrad  <G_i, g_ki>, <G_i, grad g_ki>
// then the starlet prior, dL/dh = sum_i G_i + T0, and the per-field assembly.
#include <math.h>

#include "common.cuh"
#include "corr.cuh"
#include "kernels.cuh"

namespace sr {

constexpr int kPlainTile = 64;

__global__ void plain_raster_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int epoch,
                                    float *__restrict__ fimg) {
    const FieldDev &fd = fields[0];
    const int F = fd.F, f = fd.f, M = fd.M, E = fd.E;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= F * F) return;
    const float *hpar = params + fd.param_off;
    const float *apar = hpar + (long long)F * F + (long long)epoch * M;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    const float *dpar = cpar + 2 * M + 2 * epoch;
    const int uy = u / F, ux = u - uy * F;
    float v = hpar[u];
    const float u0 = 0.5f * (float)(F - 1);
    for (int k = 0; k < M; ++k) {
        const float cx = u0 + (float)f * (cpar[2 * k] + dpar[0]);
        const float cy = u0 + (float)f * (cpar[2 * k + 1] + dpar[1]);
        const int lx = (int)floorf(cx) - kWinLo, ly = (int)floorf(cy) - kWinLo;
        if (ux >= lx && ux < lx + kWin && uy >= ly && uy < ly + kWin) {
            const float dx = src_offset(ux, F, f, cpar[2 * k], dpar[0]);
            const float dy = src_offset(uy, F, f, cpar[2 * k + 1], dpar[1]);
            v += apar[k] * (kGaussNorm * exp2f(-(dx * dx + dy * dy)));
        }
    }
    fimg[u] = v;
}

// out = S_i x (flip = 1) or S_i^T x (flip = 0) on the F x F fine grid, one 64 x 64 tile per block.
//   S:   out[u] = sum_q s[q] x[u - q + o]   -> X[i] = x[U0 - (K-1-o) + i], Kp[j] = s[K-1-j]
//   S^T: out[v] = sum_q s[q] x[v + q - o]   -> X[i] = x[V0 - o + i],       Kp[j] = s[j]
// With accumulate, out += result (running sum over epochs) and the result is also written to out2.
__global__ void __launch_bounds__(kThreads)
plain_conv_kernel(const float *__restrict__ x, const float *__restrict__ s, int F, int K, int flip,
                  float *__restrict__ out, float *__restrict__ out2) {
    extern __shared__ __align__(16) float smem[];
    const int T = kPlainTile;
    const int tiles_x = (F + T - 1) / T;
    const int ty0 = (blockIdx.x / tiles_x) * T, tx0 = (blockIdx.x % tiles_x) * T;
    const int o = K / 2;
    const int off = flip ? (K - 1 - o) : o;
    const int xrows = T + K - 1, xcols = T + K - 1, xpitch = (T + K) | 1;
    const int kpitch = (K + 3) & ~3;
    float *X = smem;
    float *Kp = smem + ((xrows * xpitch + 3) & ~3);
    for (int idx = threadIdx.x; idx < xrows * xcols; idx += blockDim.x) {
        const int i = idx / xcols, j = idx - i * xcols;
        const int gy = ty0 - off + i, gx = tx0 - off + j;
        X[i * xpitch + j] = (gy >= 0 && gy < F && gx >= 0 && gx < F) ? x[(long long)gy * F + gx] : 0.f;
    }
    for (int idx = threadIdx.x; idx < K * kpitch; idx += blockDim.x) {
        const int jy = idx / kpitch, jx = idx - jy * kpitch;
        float v = 0.f;
        if (jx < K) v = flip ? s[(K - 1 - jy) * K + (K - 1 - jx)] : s[jy * K + jx];
        Kp[idx] = v;
    }
    __syncthreads();
    const int row = threadIdx.x % T, chunk = threadIdx.x / T;  // 64 rows x 4 chunks of 16
    float acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = 0.f;
    corr_accumulate<kR>(acc, X + row * xpitch + chunk * kR, xpitch, Kp, kpitch, K);
    const int uy = ty0 + row;
    if (uy < F) {
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int ux = tx0 + chunk * kR + r;
            if (ux < F) {
                const long long q = (long long)uy * F + ux;
                if (out2) {
                    out2[q] = acc[r];
                    out[q] += acc[r];
                } else {
                    out[q] = acc[r];
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256)
plain_resid_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int epoch,
                   const float *__restrict__ conv, float *__restrict__ ebuf, double *__restrict__ chi_part,
                   double *__restrict__ se_part, int n_blocks) {
    __shared__ double s_red[2][8];
    const FieldDev &fd = fields[0];
    const int N = fd.N, f = fd.f, F = fd.F, M = fd.M, E = fd.E;
    const int p = blockIdx.x * 256 + threadIdx.x;
    const float gam = params[fd.param_off + (long long)F * F + (long long)E * M + 2 * M + 2 * E + epoch];
    double chi = 0.0, se = 0.0;
    if (p < N * N) {
        const int py = p / N, px = p - py * N;
        float mv = 0.f;
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) mv += conv[(long long)(f * py + a) * F + f * px + b];
        mv += (float)(f * f) * gam;
        const long long di = (long long)epoch * N * N + p;
        const float res = fd.d[di] - mv;
        const float wv = fd.w[di];
        chi = (double)(0.5f * wv * res * res);
        const float e = -wv * res;
        ebuf[di] = e;
        se = (double)e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        chi += __shfl_down_sync(0xffffffffu, chi, o);
        se += __shfl_down_sync(0xffffffffu, se, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = chi;
        s_red[1][threadIdx.x >> 5] = se;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += s_red[threadIdx.x][i];
        (threadIdx.x == 0 ? chi_part : se_part)[(long long)epoch * n_blocks + blockIdx.x] = s;
    }
}

__global__ void plain_up_kernel(const FieldDev *__restrict__ fields, int epoch, const float *__restrict__ ebuf,
                                float *__restrict__ ey) {
    const FieldDev &fd = fields[0];
    const int N = fd.N, f = fd.f, F = fd.F;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= F * F) return;
    const int uy = u / F, ux = u - uy * F;
    ey[u] = ebuf[(long long)epoch * N * N + (uy / f) * N + ux / f];
}

__global__ void plain_psgrad_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int epoch,
                                    const float *__restrict__ gi, float *__restrict__ ps_da,
                                    float *__restrict__ ps_du) {
    const FieldDev &fd = fields[0];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int F = fd.F, f = fd.f, M = fd.M, E = fd.E;
    if (k >= M) return;
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    const float *dpar = cpar + 2 * M + 2 * epoch;
    const float a = hpar[(long long)F * F + (long long)epoch * M + k];
    const float u0 = 0.5f * (float)(F - 1);
    const float cx = u0 + (float)f * (cpar[2 * k] + dpar[0]);
    const float cy = u0 + (float)f * (cpar[2 * k + 1] + dpar[1]);
    const int lx = (int)floorf(cx) - kWinLo, ly = (int)floorf(cy) - kWinLo;
    float sa = 0.f, sx = 0.f, sy = 0.f;
    for (int idx = lane; idx < kWin * kWin; idx += 32) {
        const int uy = ly + idx / kWin, ux = lx + idx % kWin;
        if (uy < 0 || uy >= F || ux < 0 || ux >= F) continue;
        const float dx = src_offset(ux, F, f, cpar[2 * k], dpar[0]);
        const float dy = src_offset(uy, F, f, cpar[2 * k + 1], dpar[1]);
        const float gg = gi[(long long)uy * F + ux] * (kGaussNorm * exp2f(-(dx * dx + dy * dy)));
        sa += gg;
        sx += gg * dx;
        sy += gg * dy;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        const long long s = (long long)epoch * M + k;
        ps_da[s] = sa;
        ps_du[2 * s] = a * kGaussInvSig2 * sx;
        ps_du[2 * s + 1] = a * kGaussInvSig2 * sy;
    }
}

__global__ void plain_hgrad_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ gsum,
                                   float *__restrict__ grad) {
    const FieldDev &fd = fields[0];
    const int F = fd.F;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= F * F) return;
    grad[fd.param_off + u] = gsum[u] + fd.starlet[(long long)fd.J * F * F + u];
}

static int plain_smem(int K) {
    const int T = kPlainTile;
    const int xrows = T + K - 1, xpitch = (T + K) | 1, kpitch = (K + 3) & ~3;
    return (((xrows * xpitch + 3) & ~3) + K * kpitch) * (int)sizeof(float);
}

sr_status configure_plain_kernels(int K) {
    SR_CUDA(cudaFuncSetAttribute(plain_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, plain_smem(K)));
    return SR_OK;
}

int launch_plain_eval(const FieldDev *fields, const FieldDev &hf, const float *s_raw, const ChunkItem *chunks,
                      int n_chunks, const float *params, float *grad, const PlainBuffers &pb, float *ebuf,
                      double *chi_part, double *se_part, float *ps_da, float *ps_du, const int4 *ps_items,
                      double *l1_part, double *losses, double *total, cudaStream_t st) {
    (void)ps_items;
    const int F = hf.F, K = hf.K, N = hf.N;
    const int gF = (F * F + 255) / 256;
    const int tiles = ((F + kPlainTile - 1) / kPlainTile) * ((F + kPlainTile - 1) / kPlainTile);
    const int smem = plain_smem(K);
    const int nb = (N * N + 255) / 256;
    int n = 0;
    cudaMemsetAsync(pb.gsum, 0, sizeof(float) * (size_t)F * F, st);
    for (int i = 0; i < hf.E; ++i) {
        const float *si = s_raw + (long long)i * K * K;
        plain_raster_kernel<<<gF, 256, 0, st>>>(fields, params, i, pb.fimg);
        plain_conv_kernel<<<tiles, kThreads, smem, st>>>(pb.fimg, si, F, K, 1, pb.conv, nullptr);
        plain_resid_kernel<<<nb, 256, 0, st>>>(fields, params, i, pb.conv, ebuf, chi_part, se_part, nb);
        plain_up_kernel<<<gF, 256, 0, st>>>(fields, i, ebuf, pb.ey);
        plain_conv_kernel<<<tiles, kThreads, smem, st>>>(pb.ey, si, F, K, 0, pb.gsum, pb.gi);
        if (hf.M > 0) plain_psgrad_kernel<<<1, 32 * hf.M, 0, st>>>(fields, params, i, pb.gi, ps_da, ps_du);
        n += hf.M > 0 ? 6 : 5;
    }
    const int forms = starlet_forms_single(hf.F, hf.J, hf.Wmap != nullptr);
    n += launch_starlet(fields, 1, hf.F, forms, chunks, n_chunks, hf.J, params, l1_part, st);
    plain_hgrad_kernel<<<gF, 256, 0, st>>>(fields, pb.gsum, grad);
    ++n;
    launch_finalize(fields, 1, chi_part, se_part, l1_part, ps_da, ps_du, grad, losses, total, st);
    n += 2;
    return n;
}

}  // namespace sr
