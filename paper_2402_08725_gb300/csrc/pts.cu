// Point-source prior (Eq. 11, third term) and the lambda_pts estimate of App. C.
//
// The prior lambda_pts || W o Phi^T Pbar ||_1 acts on the mean point-source image
// Pbar = sum_k <a_k> r_k, <a_k> = (1/E) sum_i a_ki, r_k the unit Gaussian of Eq. 1 at the
// source's centre c_k (no per-epoch shift).  Each field with the term active has a second
// ("shadow") FieldDev whose c_0 plane is Pbar, whose weights are lambda_pts W_j (device memory, so
// a new lambda_pts needs no new plan or graph) and whose starlet scratch is its own; the starlet
// kernels evaluate it exactly as they evaluate the prior on h.  Per evaluation:
//   pts_mean_kernel    <a_k>, FP64 sums over the epochs in order
//   pts_raster_kernel  Pbar on the fine grid (the 16 x 16 window of the tile kernels)
//   (starlet forward and adjoint levels on the shadow fields: value, and G = dP/dPbar in plane J)
//   pts_grad_kernel    per source: sum_u G r_k and <a_k> sum_u G dr_k/dc_k
// and the per-field assembly adds the value to the loss, (1/E) sum_u G r_k to every a_ki and the
// centre derivative to c_k.
//
// The estimate takes the mean epoch image fbar = (1/E) sum_i (h + sum_k a_ki r_k(c_k + delta_i)),
// h, and the unit sources r_k through the forward starlet (weighted L1 norms only) and returns
// lambda (|W o A fbar|_1 - |W o A h|_1) / sum_k <a_k> |W o A r_k|_1.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace sr {
namespace {

__device__ __forceinline__ float unit_gauss(float dx, float dy) { return kGaussNorm * exp2f(-(dx * dx + dy * dy)); }

// window of a source whose fine centre is (F - 1)/2 + f c: 16 pixels from floor(centre) - 7
__device__ __forceinline__ int win_lo(int F, int f, float c) { return (int)floorf(0.5f * (F - 1) + f * c) - kWinLo; }

__device__ __forceinline__ const float *amp_block(const FieldDev &fd, const float *params) {
    return params + fd.param_off + (long long)fd.F * fd.F;
}
__device__ __forceinline__ const float *centre_block(const FieldDev &fd, const float *params) {
    return amp_block(fd, params) + (long long)fd.E * fd.M;
}

// <a_k> for every source of every shadow field (block per shadow field)
__global__ void pts_mean_kernel(const FieldDev *__restrict__ sh, const FieldDev *__restrict__ fields,
                                const float *__restrict__ params, float *__restrict__ abar) {
    const FieldDev &sd = sh[blockIdx.x];
    const FieldDev &fd = fields[sd.pts - 1];
    const float *a = amp_block(fd, params);
    for (int k = threadIdx.x; k < fd.M; k += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < fd.E; ++i) s += (double)a[(long long)i * fd.M + k];
        abar[sd.ps_slot + k] = (float)(s / fd.E);
    }
}

// Pbar[u] = sum_k <a_k> r_k[u] on the windows; grid (pixel blocks, shadow fields)
__global__ void __launch_bounds__(256) pts_raster_kernel(const FieldDev *__restrict__ sh,
                                                         const FieldDev *__restrict__ fields,
                                                         const float *__restrict__ params,
                                                         const float *__restrict__ abar, float *__restrict__ pbar) {
    const FieldDev &sd = sh[blockIdx.y];
    const FieldDev &fd = fields[sd.pts - 1];
    const int F = fd.F, f = fd.f;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= (long long)F * F) return;
    const int uy = (int)(u / F), ux = (int)(u - (long long)uy * F);
    const float *c = centre_block(fd, params);
    float v = 0.f;
    for (int k = 0; k < fd.M; ++k) {
        const float cx = c[2 * k], cy = c[2 * k + 1];
        if ((unsigned)(ux - win_lo(F, f, cx)) < (unsigned)kWin && (unsigned)(uy - win_lo(F, f, cy)) < (unsigned)kWin)
            v += abar[sd.ps_slot + k] * unit_gauss(src_offset(ux, F, f, cx, 0.f), src_offset(uy, F, f, cy, 0.f));
    }
    pbar[sd.param_off + u] = v;
}

// One warp per source: (sum_u G r_k, <a_k> sum_u G dr_k/dc_kx, ... y) with G = T0 of the shadow's
// starlet and dr/dc = 2 ln 2 f (u - centre) r.
__global__ void pts_grad_kernel(const FieldDev *__restrict__ sh, const FieldDev *__restrict__ fields,
                                const float *__restrict__ params, const float *__restrict__ abar,
                                float *__restrict__ pts_g) {
    const FieldDev &sd = sh[blockIdx.x];
    const FieldDev &fd = fields[sd.pts - 1];
    const int F = fd.F, f = fd.f, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float *G = sd.starlet + (long long)sd.J * F * F;
    const float *c = centre_block(fd, params);
    for (int k = threadIdx.x >> 5; k < fd.M; k += nw) {
        const float cx = c[2 * k], cy = c[2 * k + 1];
        const int x0 = win_lo(F, f, cx), y0 = win_lo(F, f, cy);
        float sa = 0.f, sx = 0.f, sy = 0.f;
        for (int idx = lane; idx < kWin * kWin; idx += 32) {
            const int uy = y0 + idx / kWin, ux = x0 + idx % kWin;
            if (uy < 0 || uy >= F || ux < 0 || ux >= F) continue;
            const float dx = src_offset(ux, F, f, cx, 0.f), dy = src_offset(uy, F, f, cy, 0.f);
            const float gg = G[(long long)uy * F + ux] * unit_gauss(dx, dy);
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
            const float s = abar[sd.ps_slot + k] * kGaussInvSig2 * (float)f;
            pts_g[3 * (sd.ps_slot + k)] = sa;
            pts_g[3 * (sd.ps_slot + k) + 1] = s * sx;
            pts_g[3 * (sd.ps_slot + k) + 2] = s * sy;
        }
    }
}

// ---- estimate (App. C) ------------------------------------------------------------------

// images [2 + M][F][F]: 0 = fbar, 1 = h, 2 + k = unit r_k at c_k
__global__ void __launch_bounds__(256) est_images_kernel(FieldDev fd, const float *__restrict__ params,
                                                         float *__restrict__ img) {
    const int F = fd.F, f = fd.f, E = fd.E, M = fd.M;
    const long long FF = (long long)F * F;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= FF) return;
    const int uy = (int)(u / F), ux = (int)(u - (long long)uy * F);
    const int which = blockIdx.y;
    const float *h = params + fd.param_off, *a = amp_block(fd, params), *c = centre_block(fd, params);
    const float *dl = c + 2 * M;
    float v;
    if (which == 0) {
        double s = 0.0;
        for (int i = 0; i < E; ++i)
            for (int k = 0; k < M; ++k) {
                const float cx = c[2 * k], cy = c[2 * k + 1], ex = dl[2 * i], ey = dl[2 * i + 1];
                const int x0 = (int)floorf(0.5f * (F - 1) + f * (cx + ex)) - kWinLo;
                const int y0 = (int)floorf(0.5f * (F - 1) + f * (cy + ey)) - kWinLo;
                if ((unsigned)(ux - x0) < (unsigned)kWin && (unsigned)(uy - y0) < (unsigned)kWin)
                    s += (double)a[(long long)i * M + k] *
                         (double)unit_gauss(src_offset(ux, F, f, cx, ex), src_offset(uy, F, f, cy, ey));
            }
        v = (float)((double)h[u] + s / E);
    } else if (which == 1) {
        v = h[u];
    } else {
        const int k = which - 2;
        const float cx = c[2 * k], cy = c[2 * k + 1];
        v = ((unsigned)(ux - win_lo(F, f, cx)) < (unsigned)kWin && (unsigned)(uy - win_lo(F, f, cy)) < (unsigned)kWin)
                ? unit_gauss(src_offset(ux, F, f, cx, 0.f), src_offset(uy, F, f, cy, 0.f))
                : 0.f;
    }
    img[which * FF + u] = v;
}

constexpr float kB0 = 0.0625f, kB1 = 0.25f, kB2 = 0.375f;  // B3 spline (1,4,6,4,1)/16

__device__ __forceinline__ int refl(int t, int F) { return t < 0 ? -t : (t > F - 1 ? 2 * (F - 1) - t : t); }

__global__ void __launch_bounds__(256) est_row_kernel(const float *__restrict__ c, float *__restrict__ t, int F,
                                                      int step, long long total) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int x = (int)(idx % F);
    const float *row = c + (idx - x);
    t[idx] = kB0 * (row[refl(x - 2 * step, F)] + row[refl(x + 2 * step, F)]) +
             kB1 * (row[refl(x - step, F)] + row[refl(x + step, F)]) + kB2 * row[x];
}

// column pass in place and |w| summed per block: part[(img * (J-1) + j) * nblk + block]
__global__ void __launch_bounds__(256) est_col_l1_kernel(float *__restrict__ c, const float *__restrict__ t, int F,
                                                         int step, int j, int J1, int nblk, double *__restrict__ part) {
    __shared__ double red[256];
    const long long FF = (long long)F * F;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int img = blockIdx.y;
    double s = 0.0;
    if (u < FF) {
        const int y = (int)(u / F), x = (int)(u - (long long)y * F);
        const float *tb = t + img * FF;
        const float cn = kB0 * (tb[(long long)refl(y - 2 * step, F) * F + x] + tb[(long long)refl(y + 2 * step, F) * F + x]) +
                         kB1 * (tb[(long long)refl(y - step, F) * F + x] + tb[(long long)refl(y + step, F) * F + x]) +
                         kB2 * tb[u];
        float *cb = c + img * FF + u;
        s = fabs((double)(*cb - cn));
        *cb = cn;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[((long long)img * J1 + j) * nblk + blockIdx.x] = red[0];
}

__global__ void est_final_kernel(FieldDev fd, const float *__restrict__ params, const float *__restrict__ Wd,
                                 float lambda, const double *__restrict__ part, int nblk, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int J1 = fd.J - 1, M = fd.M, E = fd.E;
    auto wl1 = [&](int img) {
        double t = 0.0;
        for (int j = 0; j < J1; ++j) {
            double s = 0.0;
            for (int b = 0; b < nblk; ++b) s += part[((long long)img * J1 + j) * nblk + b];
            t += (double)Wd[j] * s;
        }
        return t;
    };
    const float *a = amp_block(fd, params);
    double den = 0.0;
    for (int k = 0; k < M; ++k) {
        double ab = 0.0;
        for (int i = 0; i < E; ++i) ab += (double)a[(long long)i * M + k];
        den += ab / E * wl1(2 + k);
    }
    out[0] = den != 0.0 ? (double)lambda * (wl1(0) - wl1(1)) / den : 0.0;
}

}  // namespace

int launch_pts_prior(const FieldDev *sh, const FieldDev *fields, int n_sh, int Fmax, int Mmax, int starlet_forms,
                     const ChunkItem *chunks, int n_chunks, int Jmax, const float *params, float *abar, float *pbar,
                     double *l1_pts, float *pts_g, cudaStream_t st) {
    pts_mean_kernel<<<n_sh, 64, 0, st>>>(sh, fields, params, abar);
    const long long FF = (long long)Fmax * Fmax;
    pts_raster_kernel<<<dim3((unsigned)((FF + 255) / 256), n_sh), 256, 0, st>>>(sh, fields, params, abar, pbar);
    int n = 2 + launch_starlet(sh, n_sh, Fmax, starlet_forms, chunks, n_chunks, Jmax, pbar, l1_pts, st);
    pts_grad_kernel<<<n_sh, 32 * std::min(std::max(Mmax, 1), 8), 0, st>>>(sh, fields, params, abar, pts_g);
    return n + 1;
}

sr_status pts_estimate(const FieldDev &fd, const float *params, const float *Wd, float lambda, double *out_host,
                       cudaStream_t st) {
    const int F = fd.F, n_img = 2 + fd.M, J1 = fd.J - 1;
    const long long FF = (long long)F * F;
    const int nblk = (int)((FF + 255) / 256);
    float *img = nullptr, *tmp = nullptr;
    double *part = nullptr, *out = nullptr;
    auto cleanup = [&]() {
        cudaFree(img);
        cudaFree(tmp);
        cudaFree(part);
        cudaFree(out);
    };
    cudaError_t e = cudaMalloc(&img, sizeof(float) * n_img * FF);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(float) * n_img * FF);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * (size_t)n_img * J1 * nblk);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        set_error("lambda_pts estimate: device allocation failed: %s", cudaGetErrorString(e));
        return SR_ERR_OOM;
    }
    est_images_kernel<<<dim3((unsigned)nblk, n_img), 256, 0, st>>>(fd, params, img);
    const long long total = n_img * FF;
    for (int j = 0; j < J1; ++j) {
        est_row_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(img, tmp, F, 1 << j, total);
        est_col_l1_kernel<<<dim3((unsigned)nblk, n_img), 256, 0, st>>>(img, tmp, F, 1 << j, j, J1, nblk, part);
    }
    est_final_kernel<<<1, 32, 0, st>>>(fd, params, Wd, lambda, part, nblk, out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "lambda_pts estimate");
    return SR_OK;
}

}  // namespace sr
