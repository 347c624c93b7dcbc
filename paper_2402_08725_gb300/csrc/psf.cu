// PSF reconstruction: loss (Eq. 7) and gradient kernels (sm_103a).
//
// Narrow PSF (Eq. 2): s = m(alpha, beta) + b on the F x F fine grid, m the isotropic unit-flux
// Moffat centred on pixel (F/2, F/2).  Star k (Eq. 3): t_k = D(a_k (s * r_k)) with r_k the
// 2-pixel-FWHM Gaussian shifted by shat_k = (F-1)/2 + f c_k - F/2.  The 2-D Gaussian factorises
// exactly into 1-D factors g1, so the blur is a row pass then a column pass (taps |t| <= 8,
// beyond which g1 < 2^-64 g1(0)).  The chi^2 of Eq. 4 uses diagonal weights w = 1/sigma^2.
//
// Launch sequence (all stars of the fit in each launch):
//   build_s   s = m + b
//   row       per (star, row, col): tmp0 = sum_vx s g1(t),  tmp1 = sum_vx s g1(t) t / sigma^2
//   col_fwd   per (star, data pixel): blur and its shift derivatives on the f x f block, D,
//             residual, chi^2, e = -w r, and <e, D blur>, <e, D dblur/dshift>  (FP64 partials)
//   adj_col   z = (column pass)^T D^T e
//   adj_row   gs_k = a_k (row pass)^T z               (= a_k B_k^T D^T e_k)
//   starlet   prior on b (starlet.cu)
//   reduce    dL/db = sum_k gs_k + T0, and the alpha/beta partials <sum_k gs_k, dm/dtheta>
//   finalize  loss, da_k, dc_k, dalpha, dbeta
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sr {

__device__ __forceinline__ float g1(float t) { return kGauss1Norm * exp2f(-t * t); }

__device__ __forceinline__ float2 star_shift(const FieldDev &fd, const float *params, int k) {
    const int F = fd.F;
    const float *c = params + fd.param_off + (long long)F * F + 2 + fd.E + 2 * k;
    const float base = 0.5f * (float)(F - 1) - (float)(F / 2);
    return make_float2(base + (float)fd.f * c[0], base + (float)fd.f * c[1]);
}

__device__ __forceinline__ int ceil_f(float v) { return (int)ceilf(v); }
__device__ __forceinline__ int floor_f(float v) { return (int)floorf(v); }

__global__ void psf_build_s_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params) {
    const FieldDev &fd = fields[0];
    const int F = fd.F;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= F * F) return;
    const float *b = params + fd.param_off;
    const float alpha = b[(long long)F * F], beta = b[(long long)F * F + 1];
    const int cen = F / 2;
    const int uy = u / F, ux = u - uy * F;
    const float rho2 = (float)((ux - cen) * (ux - cen) + (uy - cen) * (uy - cen));
    const float B = 1.f + rho2 / (alpha * alpha);
    const float m = (beta - 1.f) / (3.14159265358979f * alpha * alpha) * powf(B, -beta);
    fd.psf_s[u] = m + b[u];
}

__global__ void psf_row_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params) {
    const FieldDev &fd = fields[0];
    const int F = fd.F;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)fd.E * F * F) return;
    const int k = (int)(idx / ((long long)F * F));
    const int rr = (int)(idx - (long long)k * F * F);
    const int vy = rr / F, ux = rr - vy * F;
    const float sx = star_shift(fd, params, k).x;
    const float *srow = fd.psf_s + (long long)vy * F;
    int lo = ceil_f((float)ux - sx - (float)kBlurHalf), hi = floor_f((float)ux - sx + (float)kBlurHalf);
    lo = max(lo, 0);
    hi = min(hi, F - 1);
    float a0 = 0.f, a1 = 0.f;
    for (int vx = lo; vx <= hi; ++vx) {
        const float t = (float)(ux - vx) - sx;
        const float gv = srow[vx] * g1(t);
        a0 += gv;
        a1 += gv * t;
    }
    float *tmp = fd.psf_tmp + (long long)k * 3 * F * F;
    tmp[rr] = a0;
    tmp[(long long)F * F + rr] = a1 * kGaussInvSig2;
}

__global__ void __launch_bounds__(256)
psf_col_fwd_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, float *__restrict__ ebuf,
                   double *__restrict__ star_part, int n_dchunks) {
    __shared__ double s_red[4][8];
    const FieldDev &fd = fields[0];
    const int F = fd.F, N = fd.N, f = fd.f;
    const int k = blockIdx.y, chunk = blockIdx.x;
    const int p = chunk * 256 + threadIdx.x;
    const float2 sh = star_shift(fd, params, k);
    const float a = params[fd.param_off + (long long)F * F + 2 + k];
    const float *tmp0 = fd.psf_tmp + (long long)k * 3 * F * F;
    const float *tmp1 = tmp0 + (long long)F * F;
    double chi = 0.0, da = 0.0, dcx = 0.0, dcy = 0.0;
    if (p < N * N) {
        const int py = p / N, px = p - py * N;
        float mb = 0.f, bx = 0.f, by = 0.f;
        for (int ay = 0; ay < f; ++ay) {
            const int uy = f * py + ay;
            int lo = ceil_f((float)uy - sh.y - (float)kBlurHalf), hi = floor_f((float)uy - sh.y + (float)kBlurHalf);
            lo = max(lo, 0);
            hi = min(hi, F - 1);
            for (int ax = 0; ax < f; ++ax) {
                const int ux = f * px + ax;
                for (int vy = lo; vy <= hi; ++vy) {
                    const float t = (float)(uy - vy) - sh.y;
                    const float gv = g1(t);
                    const float t0 = tmp0[(long long)vy * F + ux];
                    mb += t0 * gv;
                    bx += tmp1[(long long)vy * F + ux] * gv;
                    by += t0 * gv * t;
                }
            }
        }
        by *= kGaussInvSig2;
        const long long di = (long long)k * N * N + p;
        const float res = __ldg(fd.d + di) - a * mb;
        const float wv = __ldg(fd.w + di);
        chi = (double)(0.5f * wv * res * res);
        const float e = -wv * res;
        ebuf[di] = e;
        da = (double)(e * mb);
        dcx = (double)(e * bx);
        dcy = (double)(e * by);
    }
    double v[4] = {chi, da, dcx, dcy};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) s_red[q][threadIdx.x >> 5] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += s_red[threadIdx.x][i];
        star_part[((long long)k * n_dchunks + chunk) * 4 + threadIdx.x] = s;
    }
}

__global__ void psf_adj_col_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                                   const float *__restrict__ ebuf) {
    const FieldDev &fd = fields[0];
    const int F = fd.F, N = fd.N, f = fd.f;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)fd.E * F * F) return;
    const int k = (int)(idx / ((long long)F * F));
    const int rr = (int)(idx - (long long)k * F * F);
    const int vy = rr / F, ux = rr - vy * F;
    const float sy = star_shift(fd, params, k).y;
    int lo = ceil_f((float)vy + sy - (float)kBlurHalf), hi = floor_f((float)vy + sy + (float)kBlurHalf);
    lo = max(lo, 0);
    hi = min(hi, F - 1);
    const float *e = ebuf + (long long)k * N * N + ux / f;
    float acc = 0.f;
    for (int uy = lo; uy <= hi; ++uy) acc += g1((float)(uy - vy) - sy) * e[(long long)(uy / f) * N];
    fd.psf_tmp[(long long)k * 3 * F * F + 2LL * F * F + rr] = acc;
}

__global__ void psf_adj_row_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params) {
    const FieldDev &fd = fields[0];
    const int F = fd.F;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)fd.E * F * F) return;
    const int k = (int)(idx / ((long long)F * F));
    const int rr = (int)(idx - (long long)k * F * F);
    const int vy = rr / F, vx = rr - vy * F;
    const float sx = star_shift(fd, params, k).x;
    const float a = params[fd.param_off + (long long)F * F + 2 + k];
    int lo = ceil_f((float)vx + sx - (float)kBlurHalf), hi = floor_f((float)vx + sx + (float)kBlurHalf);
    lo = max(lo, 0);
    hi = min(hi, F - 1);
    const float *z = fd.psf_tmp + (long long)k * 3 * F * F + 2LL * F * F + (long long)vy * F;
    float acc = 0.f;
    for (int ux = lo; ux <= hi; ++ux) acc += g1((float)(ux - vx) - sx) * z[ux];
    fd.psf_gs[(long long)k * F * F + rr] = a * acc;
}

__global__ void __launch_bounds__(256)
psf_reduce_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, float *__restrict__ grad,
                  double *__restrict__ ab_part) {
    __shared__ double s_red[2][8];
    const FieldDev &fd = fields[0];
    const int F = fd.F;
    const int u = blockIdx.x * 256 + threadIdx.x;
    double pa = 0.0, pb = 0.0;
    if (u < F * F) {
        double gs = 0.0;
        for (int k = 0; k < fd.E; ++k) gs += (double)fd.psf_gs[(long long)k * F * F + u];
        const float *T0 = fd.starlet + (long long)fd.J * F * F;
        grad[fd.param_off + u] = (float)(gs + (double)T0[u]);
        const float *b = params + fd.param_off;
        const float alpha = b[(long long)F * F], beta = b[(long long)F * F + 1];
        const int cen = F / 2;
        const int uy = u / F, ux = u - uy * F;
        const float rho2 = (float)((ux - cen) * (ux - cen) + (uy - cen) * (uy - cen));
        const float B = 1.f + rho2 / (alpha * alpha);
        const float m = (beta - 1.f) / (3.14159265358979f * alpha * alpha) * powf(B, -beta);
        const float dma = m * (-2.f / alpha + 2.f * beta * rho2 / (alpha * alpha * alpha * B));
        const float dmb = m * (1.f / (beta - 1.f) - logf(B));
        pa = gs * (double)dma;
        pb = gs * (double)dmb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pa += __shfl_down_sync(0xffffffffu, pa, o);
        pb += __shfl_down_sync(0xffffffffu, pb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = pa;
        s_red[1][threadIdx.x >> 5] = pb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += s_red[threadIdx.x][i];
        ab_part[2LL * blockIdx.x + threadIdx.x] = s;
    }
}

__global__ void psf_finalize_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                                    float *__restrict__ grad, const double *__restrict__ star_part, int n_dchunks,
                                    const double *__restrict__ ab_part, int n_chunks,
                                    const double *__restrict__ l1_part, double *__restrict__ losses,
                                    double *__restrict__ total) {
    const FieldDev &fd = fields[0];
    const int F = fd.F, S = fd.E, f = fd.f;
    const float *a = params + fd.param_off + (long long)F * F + 2;
    float *g = grad + fd.param_off + (long long)F * F;
    // stars: one thread each
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        double da = 0.0, dx = 0.0, dy = 0.0;
        for (int c = 0; c < n_dchunks; ++c) {
            const double *sp = star_part + ((long long)k * n_dchunks + c) * 4;
            da += sp[1];
            dx += sp[2];
            dy += sp[3];
        }
        g[2 + k] = (float)da;
        g[2 + S + 2 * k] = (float)((double)f * (double)a[k] * dx);
        g[2 + S + 2 * k + 1] = (float)((double)f * (double)a[k] * dy);
    }
    if (threadIdx.x == 0) {
        double chi = 0.0, l1 = 0.0, ga = 0.0, gb = 0.0;
        for (long long c = 0; c < (long long)S * n_dchunks; ++c) chi += star_part[4 * c];
        for (long long c = 0; c < (long long)(fd.J - 1) * fd.n_chunks; ++c) l1 += l1_part[fd.l1_slot + c];
        for (int c = 0; c < n_chunks; ++c) {
            ga += ab_part[2 * c];
            gb += ab_part[2 * c + 1];
        }
        g[0] = (float)ga;
        g[1] = (float)gb;
        losses[0] = chi + l1;
        *total = chi + l1;
    }
}

void launch_psf_model(const FieldDev *fields, int F, const float *params, cudaStream_t st) {
    psf_build_s_kernel<<<(F * F + 255) / 256, 256, 0, st>>>(fields, params);
}

int launch_psf_eval(const FieldDev *fields, const FieldDev &hf, const ChunkItem *chunks, int n_chunks,
                    const float *params, float *grad, const PsfBuffers &pb, double *l1_part, double *losses,
                    double *total, cudaStream_t st) {
    const int F = hf.F;
    const long long nst = (long long)hf.E * F * F;
    const int gF = (F * F + 255) / 256;
    const int gS = (int)((nst + 255) / 256);
    int n = 0;
    psf_build_s_kernel<<<gF, 256, 0, st>>>(fields, params); ++n;
    psf_row_kernel<<<gS, 256, 0, st>>>(fields, params); ++n;
    psf_col_fwd_kernel<<<dim3(pb.n_dchunks, hf.E), 256, 0, st>>>(fields, params, pb.ebuf, pb.star_part,
                                                                 pb.n_dchunks); ++n;
    psf_adj_col_kernel<<<gS, 256, 0, st>>>(fields, params, pb.ebuf); ++n;
    psf_adj_row_kernel<<<gS, 256, 0, st>>>(fields, params); ++n;
    const int forms = starlet_forms_single(hf.F, hf.J, hf.Wmap != nullptr);
    n += launch_starlet(fields, 1, hf.F, forms, chunks, n_chunks, hf.J, params, l1_part, st);
    psf_reduce_kernel<<<gF, 256, 0, st>>>(fields, params, grad, pb.ab_part); ++n;
    psf_finalize_kernel<<<1, 256, 0, st>>>(fields, params, grad, pb.star_part, pb.n_dchunks, pb.ab_part, gF,
                                           l1_part, losses, total); ++n;
    return n;
}

}  // namespace sr
