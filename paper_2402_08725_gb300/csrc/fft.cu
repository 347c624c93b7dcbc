// Frequency-domain form of the deconvolution loss and gradient (sm_103a).
//
// The D-folded polyphase model (deconv.cu) is a sum over phases phi of ordinary 2-D
// convolutions on the data grid, M_i = sum_phi kappa_{i,phi} * F_phi, and the adjoint is a
// correlation per phase, G_{i,phi} = kappa_{i,phi} (corr) e_i.  With circular transforms of size
// L x L, L >= N + max(tau_hi, -tau_lo), the wrap-around never reaches the N x N output, so
//     M_i = IDFT( sum_phi Khat_{i,phi} . (Hhat_phi + Phat_{i,phi}) ) on [0,N)^2,
//     G_{i,phi} = IDFT( conj(Khat_{i,phi}) . ehat_i ) on [0,N)^2,
// exactly (up to rounding).  Khat (the transforms of the folded kernels placed at tau mod L) are
// computed once per set_psfs; Hhat (the phase images of h) once per evaluation and field; the
// point sources' transforms are outer products of 1-D DFTs (the truncated, sampled Gaussian is
// separable).  Per epoch that is 2 + f^2 real 2-D transforms instead of (K+f-1)^2 taps per data
// pixel and direction.
//
// The adjoint is not transformed back per epoch: dL/dh_phi = IDFT( sum_i conj(Khat_{i,phi}) ehat_i )
// is accumulated in the frequency domain (per chunk of epochs, then per field in a fixed order)
// and transformed once per field and phase.  The point sources' gradients come from Parseval's
// identity, <G_{i,phi}, g> = L^-2 sum_k Ghat(k) conj(ghat(k)), with the separable spectra of the
// window profile and of its shift derivatives.  Per epoch that is 2 real 2-D transforms.
//
// This file holds the per-field and per-PSF kernels (Khat, Hhat, and the final dL/dh); the
// per-epoch chunk kernel, where the time goes, is in fft_fixed.cu (compile-time sizes).
//
// Transforms here: Stockham auto-sort mixed-radix FFT (radices 4, 2, 3, 5), ping-ponging between
// two shared-memory buffers, twiddles from a table exp(-2 pi i n / L).  A real L x L image is
// transformed as L/2 complex rows (two real rows per complex row), split into the half spectrum
// (L rows x L/2+1 columns), then L/2+1 complex column transforms; the inverse runs the same steps
// backwards.  Rows that are known to be zero are skipped.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace sr {

// Passed by value: the radices are packed 4 bits per stage so that nothing here is indexed at
// run time (a runtime-indexed array would put the whole struct in local memory).
struct FftGeom {
    int L, H, Lp;      // transform size, half-spectrum width L/2+1, pitch of the row-pair layout (L+1)
    int nst;
    unsigned rad;      // radix of stage s in bits [4s, 4s+4)
    const float2 *tw;  // exp(-2 pi i n / L), n < L (shared memory)
};

// y_q = sum_r v_r exp(-+ 2 pi i q r / R) for R in {2, 3, 4, 5}; s = -1 forward, +1 inverse.
__device__ __forceinline__ void small_dft(float2 *v, int R, float s) {
    if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const float2 c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        // multiplying d by s*i: (x, y) -> (-s y, s x)
        const float2 di = make_float2(-s * d.y, s * d.x);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, di);
        v[3] = csub(b, di);
    } else if (R == 3) {
        const float c1 = -0.5f, s1 = s * 0.866025403784438647f;  // cos, +-sin of 2 pi / 3
        const float2 a = v[0], b = v[1], c = v[2];
        const float2 t = cadd(b, c), u = csub(b, c);
        v[0] = cadd(a, t);
        const float2 m = make_float2(a.x + c1 * t.x, a.y + c1 * t.y);
        const float2 n = make_float2(-s1 * u.y, s1 * u.x);
        v[1] = cadd(m, n);
        v[2] = csub(m, n);
    } else {  // R == 5
        const float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;  // cos 2pi/5, cos 4pi/5
        const float s1 = s * 0.951056516295153572f, s2 = s * 0.587785252292473129f;  // sin 2pi/5, sin 4pi/5
        const float2 a = v[0];
        const float2 t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
        const float2 t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
        v[0] = make_float2(a.x + t1.x + t2.x, a.y + t1.y + t2.y);
        const float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
        const float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
        // i*(s1 u1 + s2 u2) and i*(s2 u1 - s1 u2)
        const float2 n1 = make_float2(-(s1 * u1.y + s2 * u2.y), s1 * u1.x + s2 * u2.x);
        const float2 n2 = make_float2(-(s2 * u1.y - s1 * u2.y), s2 * u1.x - s1 * u2.x);
        v[1] = cadd(m1, n1);
        v[4] = csub(m1, n1);
        v[2] = cadd(m2, n2);
        v[3] = csub(m2, n2);
    }
}

// ntr independent length-L transforms; element n of transform t at base + t*tstride + n*estride.
// Returns the buffer that holds the result (src or dst).  Warps take butterflies, lanes take
// transforms, so the twiddles of a butterfly are loaded once per warp.
__device__ float2 *stockham(float2 *src, float2 *dst, int ntr, int tstride, int estride, const FftGeom g, bool inv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float s = inv ? 1.f : -1.f;
    int Ns = 1;
    for (int st = 0; st < g.nst; ++st) {
        const int R = (int)((g.rad >> (4 * st)) & 15u);
        const int nb = g.L / R;
        const int step = g.L / (Ns * R);
        for (int j = warp; j < nb; j += nw) {
            const int k = j % Ns;
            const int obase = (j / Ns) * Ns * R + k;
            float2 w[5];
#pragma unroll
            for (int r = 1; r < 5; ++r) {
                if (r < R) {
                    const float2 t = g.tw[r * k * step];  // r k step < L
                    w[r] = inv ? conjf2(t) : t;
                }
            }
            for (int t = lane; t < ntr; t += 32) {
                const float2 *sp = src + t * tstride;
                float2 *dp = dst + t * tstride;
                float2 v[5];
                v[0] = sp[j * estride];
#pragma unroll
                for (int r = 1; r < 5; ++r)
                    if (r < R) v[r] = cmul(sp[(j + r * nb) * estride], w[r]);
                small_dft(v, R, s);
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (q < R) dp[(obase + q * Ns) * estride] = v[q];
            }
        }
        __syncthreads();
        float2 *x = src;
        src = dst;
        dst = x;
        Ns *= R;
    }
    return src;
}

// Forward real 2-D transform.  `in` holds np row pairs (row 2p in .x, row 2p+1 in .y), pitch
// Lp; rows >= 2 np are zero.  Returns the buffer with the half spectrum (pitch H).
__device__ float2 *fwd2d(float2 *in, float2 *tmp, const FftGeom g, int np) {
    float2 *r = stockham(in, tmp, np, g.Lp, 1, g, false);
    float2 *o = (r == in) ? tmp : in;
    const int L = g.L, H = g.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int y = warp; y < L; y += nw) {
        float2 *orow = o + y * H;
        if (y >= 2 * np) {
            for (int kx = lane; kx < H; kx += 32) orow[kx] = make_float2(0.f, 0.f);
            continue;
        }
        const float2 *row = r + (y >> 1) * g.Lp;
        const bool odd = y & 1;
        for (int kx = lane; kx < H; kx += 32) {
            const float2 a = row[kx];
            const float2 b = conjf2(row[kx == 0 ? 0 : L - kx]);
            orow[kx] = odd ? make_float2(0.5f * (a.y - b.y), -0.5f * (a.x - b.x))   // (a - b) / (2i)
                           : make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));   // (a + b) / 2
        }
    }
    __syncthreads();
    return stockham(o, r, H, 1, H, g, false);
}

// Inverse real 2-D transform of the half spectrum in `in` (pitch H).  Returns the buffer with
// np row pairs (pitch Lp) of the unscaled real image (multiply by 1/L^2).
__device__ float2 *inv2d(float2 *in, float2 *tmp, const FftGeom g, int np) {
    float2 *c = stockham(in, tmp, g.H, 1, g.H, g, true);
    float2 *o = (c == in) ? tmp : in;
    const int L = g.L, H = g.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = warp; p < np; p += nw) {
        const float2 *r1 = c + (2 * p) * H, *r2 = c + (2 * p + 1) * H;
        float2 *orow = o + p * g.Lp;
        for (int kx = lane; kx < L; kx += 32) {
            float2 z;
            if (kx < H) {
                const float2 a = r1[kx], b = r2[kx];
                z = make_float2(a.x - b.y, a.y + b.x);           // a + i b
            } else {
                const float2 a = r1[L - kx], b = r2[L - kx];
                z = make_float2(a.x + b.y, -a.y + b.x);          // conj(a) + i conj(b)
            }
            orow[kx] = z;
        }
    }
    __syncthreads();
    return stockham(o, c, np, g.Lp, 1, g, true);
}

__device__ __forceinline__ void load_geom(FftGeom &g, const FieldDev &fd, float2 *tw_smem) {
    g.L = fd.fft_L;
    g.H = fd.fft_L / 2 + 1;
    g.Lp = fd.fft_L + 1;
    g.nst = fd.fft_nst;
    g.rad = 0u;
#pragma unroll
    for (int s = 0; s < kFftMaxStages; ++s) g.rad |= (unsigned)(fd.fft_rad[s] & 15) << (4 * s);
    for (int n = threadIdx.x; n < g.L; n += blockDim.x) tw_smem[n] = fd.fft_tw[n];
    g.tw = tw_smem;
}

// ---------------------------------------------------------------------------------------------
// Hhat_phi: transforms of the phase images of h, F_phi[m] = h[f m + phi].  One block per
// (fft field, phi): blockIdx.y indexes fft_fields[] (costliest fields first), blockIdx.x is phi.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFftThreads)
fft_hhat_kernel(const FieldDev *__restrict__ fields, const int *__restrict__ fft_fields,
                const float *__restrict__ params, float2 *__restrict__ hhat_all) {
    extern __shared__ __align__(16) float2 fsm[];
    const FieldDev &fd = fields[fft_fields[blockIdx.y]];
    const int f = fd.f, N = fd.N, F = fd.F, nph = f * f;
    const int ph = blockIdx.x;
    if (ph >= nph) return;
    const int L = fd.fft_L, H = L / 2 + 1, Lp = L + 1;
    float2 *A = fsm, *B = fsm + L * H, *tw = fsm + 2 * L * H;
    FftGeom g;
    load_geom(g, fd, tw);
    const int phy = ph / f, phx = ph - phy * f;
    const float *h = params + fd.param_off;
    const int np = (N + 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = warp; p < np; p += nw) {
        for (int x = lane; x < L; x += 32) {
            float v[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int y = 2 * p + q;
                v[q] = (y < N && x < N) ? h[(long long)(f * y + phy) * F + f * x + phx] : 0.f;
            }
            A[p * Lp + x] = make_float2(v[0], v[1]);
        }
    }
    __syncthreads();
    float2 *S = fwd2d(A, B, g, np);
    const int Hp = H + 1;  // global row pitch (pad column zero)
    float2 *out = hhat_all + fd.fft_hhat_off + (long long)ph * L * Hp;
    for (int idx = threadIdx.x; idx < L * Hp; idx += blockDim.x) {
        const int ky = idx / Hp, kx = idx - ky * Hp;
        out[idx] = kx < H ? S[ky * H + kx] : make_float2(0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------------------------
// dL/dh for the fft fields: sum the chunk accumulators of the field in a fixed order, transform
// back, and add the prior's gradient.  One block per (fft field, phi).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFftThreads)
fft_hgrad_kernel(const FieldDev *__restrict__ fields, const int *__restrict__ fft_fields,
                 const float2 *__restrict__ acc_all, float *__restrict__ grad) {
    extern __shared__ __align__(16) float2 fsm[];
    const FieldDev &fd = fields[fft_fields[blockIdx.y]];
    const int f = fd.f, N = fd.N, F = fd.F, nph = f * f;
    const int ph = blockIdx.x;
    if (ph >= nph) return;
    const int L = fd.fft_L, H = L / 2 + 1, Lp = L + 1, LH = L * H;
    float2 *A = fsm, *B = fsm + LH, *tw = fsm + 2 * LH;
    FftGeom g;
    load_geom(g, fd, tw);
    const int n_chunks = fd.fft_n_chunks;
    const int Hp = H + 1, LHp = L * Hp;  // global row pitch of the accumulators
    for (int idx = threadIdx.x; idx < LH; idx += blockDim.x) {
        const int ky = idx / H, kx = idx - ky * H;
        // eight interleaved partial sums (chunk c into c mod 8), combined in a fixed order: eight
        // loads in flight instead of one dependent chain
        const float2 *ac = acc_all + fd.fft_acc_off + (long long)ph * LHp + ky * Hp + kx;
        const long long cs = (long long)nph * LHp;
        float2 p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = make_float2(0.f, 0.f);
        int c = 0;
        for (; c + 8 <= n_chunks; c += 8) {
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q] = cadd(p[q], __ldg(&ac[(c + q) * cs]));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (c + q < n_chunks) p[q] = cadd(p[q], __ldg(&ac[(c + q) * cs]));
        A[idx] = cadd(cadd(cadd(p[0], p[1]), cadd(p[2], p[3])), cadd(cadd(p[4], p[5]), cadd(p[6], p[7])));
    }
    __syncthreads();
    const int np = (N + 1) / 2;
    const float2 *Gp = inv2d(A, B, g, np);
    const float scale = 1.f / ((float)L * (float)L);
    const int phy = ph / f, phx = ph - phy * f;
    const float *T0 = fd.starlet + (long long)fd.J * F * F;
    float *gh = grad + fd.param_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = warp; p < np; p += nw) {
        for (int x = lane; x < N; x += 32) {
            const float2 v = Gp[p * Lp + x];
            const int y = 2 * p;
            const long long u0 = (long long)(f * y + phy) * F + f * x + phx;
            gh[u0] = v.x * scale + T0[u0];
            if (y + 1 < N) {
                const long long u1 = u0 + (long long)f * F;
                gh[u1] = v.y * scale + T0[u1];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
int fft_smem_bytes(int L, int M, int f) {
    const int H = L / 2 + 1;
    return (2 * L * H + L + 2 * M * f * (H + L)) * (int)sizeof(float2);
}

template <typename K>
static sr_status set_dyn_smem(K kernel, int optin, int *limit) {
    cudaFuncAttributes a;
    SR_CUDA(cudaFuncGetAttributes(&a, kernel));
    const int dyn = optin - (int)a.sharedSizeBytes;
    SR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    *limit = std::min(*limit, dyn);
    return SR_OK;
}

// Opens the largest dynamic shared memory each transform kernel can take (the opt-in limit
// less its static shared memory) and returns the smallest of these in *limit.
sr_status configure_fft_kernels(int optin, int *limit) {
    *limit = optin;
    sr_status s;
    if ((s = set_dyn_smem(fft_hhat_kernel, optin, limit)) != SR_OK) return s;
    if ((s = set_dyn_smem(fft_hgrad_kernel, optin, limit)) != SR_OK) return s;
    return SR_OK;
}

void launch_fft_hhat(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_nph, int smem,
                     const float *params, float2 *hhat, cudaStream_t st) {
    fft_hhat_kernel<<<dim3(max_nph, n_fft_fields), kFftThreads, smem, st>>>(fields, fft_fields, params, hhat);
}

void launch_fft_hgrad(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_nph, int smem,
                      const float2 *acc, float *grad, cudaStream_t st) {
    fft_hgrad_kernel<<<dim3(max_nph, n_fft_fields), kFftThreads, smem, st>>>(fields, fft_fields, acc, grad);
}

}  // namespace sr
