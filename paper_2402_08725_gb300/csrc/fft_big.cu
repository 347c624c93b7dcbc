// Frequency-domain form for transforms larger than shared memory (sm_103a).
//
// A field whose wrap-free transform size L (L >= N + max(tau_hi, -tau_lo), L >= Tk) is beyond the
// in-shared-memory sizes of fft_pair.cu (a wide PSF on a large stamp: 255 x 255 PSFs on 512 x 512
// frames at f = 3 give L = 576) is transformed through global memory.  The model and its adjoint
// are the same as there (Eq. 8-10 with the block sum folded into the kernels):
//     M_e = IDFT( sum_phi Khat_{e,phi} Fhat_{e,phi} ),   dL/dh_phi = IDFT( sum_e conj(Khat_{e,phi}) ehat_e ),
// with one difference: the point sources are rasterised into each frame's fine image
// f_e = h + sum_k a_ek r_k (Eq. 9) before its phase images are transformed, so the spectra carry no
// point-source term (any number of sources); their gradients <G_{e,phi}, r_k> are taken directly on
// each source's 16 x 16 window (big_window_adj_kernel, then the direct form's psgrad_kernel).
//
// A 2-D transform is a transform of rows, a transpose, and a transform of rows again.  Each row
// transform holds kBgRows rows of L complex values in shared memory and runs the in-place
// four-step passes of fft_pair.cuh (L = R1 R2, spectra in digit-transposed order inside a row,
// natural order in global memory).  Two real images always travel together as one complex image
// (two phases of an image, or two frames), separated or joined with Hermitian symmetry on the rows
// kx and L - kx of the transposed spectrum.  Spectra are stored transposed: [kx < L/2 + 1][ky < L].
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"
#include "ffsum.cuh"
#include "fft_pair.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

__host__ __device__ constexpr int bg_r1(int L) {
    return (L == 192 || L == 240 || L == 288 || L == 384 || L == 576 || L == 768) ? 24 : 0;
}

template <int L>
struct Bg {
    static constexpr int R1 = bg_r1(L), R2 = L / R1;
    static constexpr int S = (R2 & 1) ? R2 : R2 + 1;  // physical length of a group of R2 positions
    static constexpr int RW = R1 * S;                  // physical row width (float2)
    static constexpr int H = L / 2 + 1;
    static_assert(R1 > 0 && R1 * R2 == L, "transform size not in the list");
};
constexpr int kBgRows = 8;        // rows per block of the row transforms
constexpr int kBgThreads = 192;   // threads per block of the row transforms (one per pass item)
constexpr int kBgItems = kBgRows / 2;  // (kx, L - kx) row pairs per block of the transposed-row kernels
constexpr int kBgMaxSources = 64;      // the most point sources a problem may have

// physical column of spatial position x, and of frequency k
template <int L>
__device__ __forceinline__ int bpx(int x) {
    return (x / Bg<L>::R2) * Bg<L>::S + x % Bg<L>::R2;
}
template <int L>
__device__ __forceinline__ int bpk(int k) {
    return (k % Bg<L>::R1) * Bg<L>::S + k / Bg<L>::R1;
}

// In-place forward transforms of nr rows (pitch RW): spatial x < xlim (zero beyond) to frequencies.
template <int L>
__device__ void bg_fwd(float2 *Z, int nr, int xlim, const float2 *TWL) {
    using G = Bg<L>;
    constexpr int R1 = G::R1, R2 = G::R2, S = G::S, RW = G::RW;
    for (int t = threadIdx.x; t < nr * R2; t += blockDim.x) {
        const int row = t / R2, n2 = t - row * R2;
        float2 *z = Z + row * RW + n2;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = n2 + R2 * n1 < xlim ? z[n1 * S] : make_float2(0.f, 0.f);
        dft<R1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) z[k1 * S] = k1 == 0 ? v[0] : cmul(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * R1; t += blockDim.x) {
        const int row = t / R1, k1 = t - row * R1;
        float2 *z = Z + row * RW + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = z[n2];
        dft<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) z[k2] = v[k2];
    }
    __syncthreads();
}

// In-place inverse transforms of nr rows: frequencies to spatial positions, x < xlim written.
template <int L>
__device__ void bg_inv(float2 *Z, int nr, int xlim, const float2 *TWL) {
    using G = Bg<L>;
    constexpr int R1 = G::R1, R2 = G::R2, S = G::S, RW = G::RW;
    for (int t = threadIdx.x; t < nr * R1; t += blockDim.x) {
        const int row = t / R1, k1 = t - row * R1;
        float2 *z = Z + row * RW + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = z[k2];
        dft<R2, true>(v);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) z[n2] = n2 == 0 ? v[0] : cmulc(v[n2], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * R2; t += blockDim.x) {
        const int row = t / R2, n2 = t - row * R2;
        float2 *z = Z + row * RW + n2;
        float2 v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = z[k1 * S];
        dft<R1, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
            if (n2 + R2 * n1 < xlim) z[n1 * S] = v[n1];
    }
    __syncthreads();
}

template <int L>
__device__ __forceinline__ void bg_twl(float2 *TWL, const float2 *tw) {
    constexpr int R2 = Bg<L>::R2;
    for (int n = threadIdx.x; n < L; n += blockDim.x) TWL[n] = tw[(n % R2) * (n / R2)];
}

__device__ __forceinline__ float gauss2(float dx, float dy) { return kGaussNorm * exp2f(-(dx * dx + dy * dy)); }

// ---------------------------------------------------------------------------------------------
// Row transforms of the inputs.  Image j = e * npr + q (frame e, phases 2q and 2q + 1 as the real
// and imaginary parts):
//   mode 0: the phase images of f_e = h + the frame's point sources (rows y < N, x < N);
//   mode 1: the folded kernels kappa_{e,phi} placed at tau - tau_lo (rows y < Tk, x < Tk).
// Rows [y0, y0 + kBgRows) of image blockIdx.y, transformed along x, to zb[j][y][kx].
// ---------------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(kBgThreads) big_load_rows_kernel(FieldDev fd, const float *__restrict__ params,
                                                                   int mode, float2 *__restrict__ zb, int ny) {
    using G = Bg<L>;
    extern __shared__ __align__(16) float2 bsm[];
    float2 *Z = bsm, *TWL = bsm + kBgRows * G::RW;
    __shared__ float4 s_src[kBgMaxSources];
    __shared__ int2 s_win[kBgMaxSources];
    __shared__ unsigned long long s_rowmask[kBgRows][2];  // sources whose window holds the fine row
    bg_twl<L>(TWL, fd.fft_tw);
    const int f = fd.f, N = fd.N, F = fd.F, M = fd.M, E = fd.E, nph = f * f, npr = (nph + 1) / 2;
    const int j = blockIdx.y, e = j / npr, q = j - e * npr;
    const int pa = 2 * q, pb = 2 * q + 1;
    const bool hasb = pb < nph;
    const int y0 = blockIdx.x * kBgRows;
    const int nx = mode == 0 ? N : fd.Tk;
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    const float *dpar = cpar + 2 * M + 2 * e;
    if (mode == 0 && threadIdx.x < M) {
        const int k = threadIdx.x;
        const float u0 = 0.5f * (float)(F - 1);
        const float cx = u0 + (float)f * (cpar[2 * k] + dpar[0]), cy = u0 + (float)f * (cpar[2 * k + 1] + dpar[1]);
        s_src[k] = make_float4(cpar[2 * k], cpar[2 * k + 1], hpar[(long long)F * F + (long long)e * M + k], 0.f);
        s_win[k] = make_int2((int)floorf(cx) - kWinLo, (int)floorf(cy) - kWinLo);
    }
    __syncthreads();
    if (mode == 0 && threadIdx.x < 2 * kBgRows) {
        const int r = threadIdx.x >> 1, w = threadIdx.x & 1;
        const int ph = w ? pb : pa;
        const int uy = f * (y0 + r) + ph / f;
        unsigned long long m = 0ull;
        for (int k = 0; k < M; ++k)
            if ((unsigned)(uy - s_win[k].y) < (unsigned)kWin) m |= 1ull << k;
        s_rowmask[r][w] = m;
    }
    __syncthreads();
    if (mode == 1) {
        for (int t = threadIdx.x; t < kBgRows * nx; t += blockDim.x) {
            const int r = t / nx, x = t - r * nx;
            const int y = y0 + r;
            float2 v = make_float2(0.f, 0.f);
            if (y < ny) {
                const float *ka = fd.kappa + ((long long)e * nph + pa) * fd.Tk * fd.Tk + y * fd.Tk + x;
                v = make_float2(ka[0], hasb ? ka[fd.Tk * fd.Tk] : 0.f);
            }
            Z[r * G::RW + bpx<L>(x)] = v;
        }
    } else {
        // h at the two phases first (independent loads, several in flight per thread), then the
        // point sources of the rows that have any, added in index order to the same elements by
        // the same threads
        const int pay = pa / f, pax = pa - pay * f, pby = pb / f, pbx = pb - pby * f;
#pragma unroll 4
        for (int t = threadIdx.x; t < kBgRows * nx; t += blockDim.x) {
            const int r = t / nx, x = t - r * nx;
            const int y = y0 + r;
            float2 v = make_float2(0.f, 0.f);
            if (y < ny) {
                v.x = __ldg(hpar + (long long)(f * y + pay) * F + f * x + pax);
                if (hasb) v.y = __ldg(hpar + (long long)(f * y + pby) * F + f * x + pbx);
            }
            Z[r * G::RW + bpx<L>(x)] = v;
        }
        for (int t = threadIdx.x; t < kBgRows * nx; t += blockDim.x) {
            const int r = t / nx, x = t - r * nx;
            const int y = y0 + r;
            if (y >= ny || (s_rowmask[r][0] | s_rowmask[r][1]) == 0ull) continue;
            float2 &z = Z[r * G::RW + bpx<L>(x)];
            float val[2] = {z.x, z.y};
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int ph = w ? pb : pa;
                if (w == 1 && !hasb) break;
                const int phy = ph / f, phx = ph - phy * f;
                const int uy = f * y + phy, ux = f * x + phx;
                float s = val[w];
                // the sources whose window holds the pixel, in index order
                for (unsigned long long m = s_rowmask[r][w]; m; m &= m - 1) {
                    const int k = __ffsll((long long)m) - 1;
                    if ((unsigned)(ux - s_win[k].x) < (unsigned)kWin)
                        s += s_src[k].z * gauss2(src_offset(ux, F, f, s_src[k].x, dpar[0]),
                                                 src_offset(uy, F, f, s_src[k].y, dpar[1]));
                }
                val[w] = s;
            }
            z = make_float2(val[0], val[1]);
        }
    }
    __syncthreads();
    bg_fwd<L>(Z, kBgRows, nx, TWL);
    float2 *out = zb + (long long)j * ny * L;
    for (int t = threadIdx.x; t < kBgRows * L; t += blockDim.x) {
        const int r = t / L, k = t - r * L;
        if (y0 + r < ny) out[(long long)(y0 + r) * L + k] = Z[r * G::RW + bpk<L>(k)];
    }
}

// out[j][c][r] = in[j][r][c] for r < R, c < C (32 x 32 tiles through shared memory)
__global__ void big_transpose_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int R, int C) {
    __shared__ float2 tile[32][33];
    const long long j = blockIdx.z;
    const float2 *src = in + j * R * C;
    float2 *dst = out + j * R * C;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = src[(long long)r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[(long long)c * R + r] = tile[threadIdx.x][i];
    }
}

// ---------------------------------------------------------------------------------------------
// Kernels on the transposed rows: block items kx = blockIdx.x * kBgItems + i (kx < L/2 + 1), each
// with its partner row L - kx (the same row for kx = 0 and kx = L/2).  Slot 2i holds row kx, slot
// 2i + 1 row L - kx.
// ---------------------------------------------------------------------------------------------
enum { BG_SPLIT = 0, BG_MODEL = 1, BG_ADJ = 2, BG_HJOIN = 3, BG_RESID_ROWS = 4, BG_HOUT_ROWS = 5 };

struct BgArgs {
    const float2 *zt_in;   // SPLIT, ADJ: transposed rows [image][L][ny]
    float2 *zt_out;        // MODEL, HJOIN: transposed rows [image][L][N]
    float2 *spec;          // SPLIT: output spectra [E][nph][H][L]
    const float2 *khat;    // MODEL, ADJ: kernel spectra [E][nph][H][L]
    const float2 *fhat;    // MODEL: image spectra [E][nph][H][L]
    float2 *acc;           // ADJ (write), HJOIN (read): adjoint spectra of each frame pair [pairs][nph][H][L]
    int ny;                // SPLIT, ADJ: spatial extent of the input rows
    int shift;             // SPLIT: tau_lo mod L (0: none)
    int npairs;            // HJOIN: frame pairs whose adjoint spectra are added (in order)
};

template <int L, int MODE>
__global__ void __launch_bounds__(kBgThreads) big_cols_kernel(FieldDev fd, BgArgs a) {
    using G = Bg<L>;
    constexpr int H = G::H, RW = G::RW;
    extern __shared__ __align__(16) float2 bsm[];
    float2 *Z = bsm, *TWL = bsm + kBgRows * RW;
    bg_twl<L>(TWL, fd.fft_tw);
    const int f = fd.f, N = fd.N, E = fd.E, nph = f * f, npr = (nph + 1) / 2;
    const int j = blockIdx.y;  // image (SPLIT: e * npr + q; MODEL, ADJ: frame pair; HJOIN: q)
    const int kx0 = blockIdx.x * kBgItems;
    const long long SL = (long long)H * L;  // one transposed half spectrum
    // load or build the rows
    if constexpr (MODE == BG_SPLIT || MODE == BG_ADJ) {
        const int ny = a.ny;
        const float2 *src = a.zt_in + (long long)j * L * ny;
        for (int t = threadIdx.x; t < kBgRows * ny; t += blockDim.x) {
            const int s = t / ny, y = t - s * ny;
            const int kx = kx0 + (s >> 1);
            float2 v = make_float2(0.f, 0.f);
            if (kx < H) {
                const int row = (s & 1) ? (L - kx) % L : kx;
                v = src[(long long)row * ny + y];
            }
            Z[s * RW + bpx<L>(y)] = v;
        }
        __syncthreads();
        bg_fwd<L>(Z, kBgRows, ny, TWL);
    } else {
        const int e0 = 2 * j, e1 = e0 + 1;
        const bool has1 = MODE == BG_MODEL ? e1 < E : (2 * j + 1 < nph);
        for (int t = threadIdx.x; t < kBgItems * L; t += blockDim.x) {
            const int i = t / L, ky = t - i * L;
            const int kx = kx0 + i;
            if (kx >= H) continue;
            const bool selfrow = kx == 0 || 2 * kx == L;
            if (selfrow && 2 * ky > L) continue;  // written with the conjugate of -ky
            float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
            const long long off = (long long)kx * L + ky;
            if (MODE == BG_MODEL) {
                // the loads of four phases in flight together, added in phase order
                const float2 *__restrict__ k0 = a.khat + (long long)e0 * nph * SL + off;
                const float2 *__restrict__ x0 = a.fhat + (long long)e0 * nph * SL + off;
                const float2 *__restrict__ k1 = a.khat + (long long)e1 * nph * SL + off;
                const float2 *__restrict__ x1 = a.fhat + (long long)e1 * nph * SL + off;
                for (int p0 = 0; p0 < nph; p0 += 4) {
                    float2 ka[4], xa[4], kb[4], xb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long o = (long long)(p0 + u) * SL;
                        const bool in = p0 + u < nph;
                        ka[u] = in ? __ldg(k0 + o) : make_float2(0.f, 0.f);
                        xa[u] = in ? __ldg(x0 + o) : make_float2(0.f, 0.f);
                        kb[u] = in && has1 ? __ldg(k1 + o) : make_float2(0.f, 0.f);
                        xb[u] = in && has1 ? __ldg(x1 + o) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (p0 + u >= nph) break;
                        A = cadd(A, cmul(ka[u], xa[u]));
                        if (has1) B = cadd(B, cmul(kb[u], xb[u]));
                    }
                }
            } else {  // HJOIN: phases 2j and 2j + 1, the frame pairs' adjoint spectra added in order
                for (int p = 0; p < a.npairs; ++p) {
                    const float2 *ap = a.acc + (long long)p * nph * SL;
                    A = cadd(A, ap[(long long)(2 * j) * SL + off]);
                    if (has1) B = cadd(B, ap[(long long)(2 * j + 1) * SL + off]);
                }
            }
            const int kym = (L - ky) % L;
            float2 *r0 = Z + (2 * i) * RW, *r1 = Z + (selfrow ? 2 * i : 2 * i + 1) * RW;
            if (selfrow && (ky == 0 || 2 * ky == L)) {
                r0[bpk<L>(ky)] = make_float2(A.x, B.x);
            } else {
                r0[bpk<L>(ky)] = make_float2(A.x - B.y, A.y + B.x);    // A + i B
                r1[bpk<L>(kym)] = make_float2(A.x + B.y, B.x - A.y);   // conj(A) + i conj(B)
            }
        }
        __syncthreads();
        bg_inv<L>(Z, kBgRows, N, TWL);
    }
    // use or store the rows
    if constexpr (MODE == BG_MODEL || MODE == BG_HJOIN) {
        float2 *dst = a.zt_out + (long long)j * L * N;
        for (int t = threadIdx.x; t < kBgRows * N; t += blockDim.x) {
            const int s = t / N, y = t - s * N;
            const int kx = kx0 + (s >> 1);
            if (kx >= H) continue;
            const bool selfrow = kx == 0 || 2 * kx == L;
            if ((s & 1) && selfrow) continue;
            const int row = (s & 1) ? L - kx : kx;
            dst[(long long)row * N + y] = Z[s * RW + bpx<L>(y)];
        }
    } else {
    for (int t = threadIdx.x; t < kBgItems * L; t += blockDim.x) {
        const int i = t / L, ky = t - i * L;
        const int kx = kx0 + i;
        if (kx >= H) continue;
        const bool selfrow = kx == 0 || 2 * kx == L;
        const float2 A = Z[(2 * i) * RW + bpk<L>(ky)];
        const float2 B = Z[(selfrow ? 2 * i : 2 * i + 1) * RW + bpk<L>((L - ky) % L)];
        const float2 xa = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));   // (A + conj B) / 2
        const float2 xb = make_float2(0.5f * (A.y + B.y), 0.5f * (B.x - A.x));   // (A - conj B) / 2i
        const long long off = (long long)kx * L + ky;
        if (MODE == BG_SPLIT) {
            const int e = j / npr, q = j - e * npr;
            float2 va = xa, vb = xb;
            if (a.shift) {
                const float2 w = fd.fft_tw[((ky + kx) * a.shift) % L];
                va = cmul(va, w);
                vb = cmul(vb, w);
            }
            a.spec[((long long)e * nph + 2 * q) * SL + off] = va;
            if (2 * q + 1 < nph) a.spec[((long long)e * nph + 2 * q + 1) * SL + off] = vb;
        } else {  // ADJ: the pair's acc_phi = conj(Khat_{e0,phi}) ehat_e0 + conj(Khat_{e1,phi}) ehat_e1
            const int e0 = 2 * j, e1 = e0 + 1;
            const bool has1 = e1 < E;
            float2 *__restrict__ ap = a.acc + (long long)j * nph * SL + off;
            const float2 *__restrict__ k0 = a.khat + (long long)e0 * nph * SL + off;
            const float2 *__restrict__ k1 = a.khat + (long long)e1 * nph * SL + off;
            // the kernel spectra of four phases in flight together
            for (int p0 = 0; p0 < nph; p0 += 4) {
                float2 ka[4], kb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long o = (long long)(p0 + u) * SL;
                    const bool in = p0 + u < nph;
                    ka[u] = in ? __ldg(k0 + o) : make_float2(0.f, 0.f);
                    kb[u] = in && has1 ? __ldg(k1 + o) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (p0 + u >= nph) break;
                    float2 run = cmulc(xa, ka[u]);
                    if (has1) run = cadd(run, cmulc(xb, kb[u]));
                    ap[(long long)(p0 + u) * SL] = run;
                }
            }
        }
    }
    }
}

// ---------------------------------------------------------------------------------------------
// Kernels on the image rows (y < N) of one complex image [N][L] (frequencies along x):
//   RESID: transform back along x; with m_e = Re/Im * L^-2 + f^2 Gamma_e the residual e = -w (d - m)
//          of frames 2 pair and 2 pair + 1 (e to ebuf, chi^2 and sum e per row), and e0 + i e1
//          transformed along x again;
//   HOUT:  transform back along x; dL/dh of phases 2q and 2q + 1 = Re/Im * L^-2 + the prior's part.
// ---------------------------------------------------------------------------------------------
template <int L, int MODE>
__global__ void __launch_bounds__(kBgThreads) big_rows_kernel(FieldDev fd, float2 *__restrict__ zb,
                                                              const float *__restrict__ params,
                                                              float *__restrict__ ebuf, double *__restrict__ chi_part,
                                                              double *__restrict__ se_part, float *__restrict__ grad) {
    using G = Bg<L>;
    constexpr int RW = G::RW;
    constexpr int TPR = kBgThreads / kBgRows;  // threads per row in the residual
    extern __shared__ __align__(16) float2 bsm[];
    float2 *Z = bsm, *TWL = bsm + kBgRows * RW;
    __shared__ float4 red[kBgRows][TPR];
    bg_twl<L>(TWL, fd.fft_tw);
    const int f = fd.f, N = fd.N, F = fd.F, E = fd.E, M = fd.M;
    const int j = blockIdx.y;  // RESID: frame pair; HOUT: pair of phases
    float2 *img = zb + (long long)j * N * L;
    const int y0 = blockIdx.x * kBgRows;
    for (int t = threadIdx.x; t < kBgRows * L; t += blockDim.x) {
        const int r = t / L, k = t - r * L;
        Z[r * RW + bpk<L>(k)] = y0 + r < N ? img[(long long)(y0 + r) * L + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    bg_inv<L>(Z, kBgRows, N, TWL);
    const float scale = 1.f / ((float)L * (float)L);
    if constexpr (MODE == BG_RESID_ROWS) {
        const int e0 = 2 * j, e1 = e0 + 1;
        const bool has1 = e1 < E;
        const float *gam = params + fd.param_off + (long long)F * F + (long long)E * M + 2 * M + 2 * E;
        const float bg0 = (float)(f * f) * gam[e0], bg1 = has1 ? (float)(f * f) * gam[e1] : 0.f;
        const int r = threadIdx.x / TPR, l = threadIdx.x - r * TPR;
        const int y = y0 + r;
        FSum c0 = fsum_zero(), c1 = fsum_zero(), s0 = fsum_zero(), s1 = fsum_zero();
        if (y < N) {
            const long long o0 = ((long long)e0 * N + y) * N, o1 = o0 + (long long)N * N;
            float *eb = ebuf + fd.ebuf_off;
            for (int x = l; x < N; x += TPR) {
                float2 *zp = Z + r * RW + bpx<L>(x);
                const float2 mv = *zp;
                const float d0 = fd.d[o0 + x], w0 = fd.w[o0 + x];
                const float rr0 = d0 - (mv.x * scale + bg0);
                const float ev0 = -w0 * rr0;
                c0 = fsum_add(c0, 0.5f * w0 * rr0 * rr0);
                s0 = fsum_add(s0, ev0);
                eb[o0 + x] = ev0;
                float ev1 = 0.f;
                if (has1) {
                    const float d1 = fd.d[o1 + x], w1 = fd.w[o1 + x];
                    const float rr1 = d1 - (mv.y * scale + bg1);
                    ev1 = -w1 * rr1;
                    c1 = fsum_add(c1, 0.5f * w1 * rr1 * rr1);
                    s1 = fsum_add(s1, ev1);
                    eb[o1 + x] = ev1;
                }
                *zp = make_float2(ev0, ev1);
            }
        }
        // per-row sums in a fixed order (thread 0 of the row adds its row's partials in order)
        red[r][l] = make_float4(c0.hi, c0.lo, s0.hi, s0.lo);
        __syncthreads();
        if (l == 0 && y < N) {
            FSum cc = fsum_zero(), ss = fsum_zero();
            for (int u = 0; u < TPR; ++u) {
                cc = fsum_add(cc, FSum{red[r][u].x, red[r][u].y});
                ss = fsum_add(ss, FSum{red[r][u].z, red[r][u].w});
            }
            chi_part[fd.tile_slot + (long long)e0 * N + y] = fsum_value(cc);
            se_part[fd.tile_slot + (long long)e0 * N + y] = fsum_value(ss);
        }
        __syncthreads();
        red[r][l] = make_float4(c1.hi, c1.lo, s1.hi, s1.lo);
        __syncthreads();
        if (l == 0 && y < N && has1) {
            FSum cc = fsum_zero(), ss = fsum_zero();
            for (int u = 0; u < TPR; ++u) {
                cc = fsum_add(cc, FSum{red[r][u].x, red[r][u].y});
                ss = fsum_add(ss, FSum{red[r][u].z, red[r][u].w});
            }
            chi_part[fd.tile_slot + (long long)e1 * N + y] = fsum_value(cc);
            se_part[fd.tile_slot + (long long)e1 * N + y] = fsum_value(ss);
        }
        __syncthreads();
        bg_fwd<L>(Z, kBgRows, N, TWL);
        for (int t = threadIdx.x; t < kBgRows * L; t += blockDim.x) {
            const int rr = t / L, k = t - rr * L;
            if (y0 + rr < N) img[(long long)(y0 + rr) * L + k] = Z[rr * RW + bpk<L>(k)];
        }
    } else {  // HOUT
        const int nph = f * f, pa = 2 * j, pb = pa + 1;
        const bool hasb = pb < nph;
        const int pay = pa / f, pax = pa - pay * f, pby = pb / f, pbx = pb - pby * f;
        const float *T0 = fd.starlet + (long long)fd.J * F * F;
        float *gh = grad + fd.param_off;
        for (int t = threadIdx.x; t < kBgRows * N; t += blockDim.x) {
            const int r = t / N, x = t - r * N;
            const int y = y0 + r;
            if (y >= N) continue;
            const float2 v = Z[r * RW + bpx<L>(x)];
            const long long ua = (long long)(f * y + pay) * F + f * x + pax;
            gh[ua] = v.x * scale + T0[ua];
            if (hasb) {
                const long long ub = (long long)(f * y + pby) * F + f * x + pbx;
                gh[ub] = v.y * scale + T0[ub];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The adjoint images G_{e,phi}[m] = sum_{t in [0, Tk)^2} kappa_{e,phi}[t] e_e[m + tau_lo + t] (zero
// outside the data grid: the correlation the direct form's adj_kernel computes) on the phase-phi
// positions m of source k's window, written to gbuf for psgrad_kernel.  One block per (frame,
// source, phase); the block stages kappa_{e,phi} and the e patch the window needs, and each window
// position's sum is split over groups of kernel rows that are then added in a fixed order.  Two
// sources whose windows overlap write the same value twice.
// ---------------------------------------------------------------------------------------------
constexpr int kWinThreads = 256;
constexpr int kWinRun = 6;  // window positions per thread and pass (the whole row at f = 3)

__global__ void __launch_bounds__(kWinThreads) big_window_adj_kernel(FieldDev fd, const float *__restrict__ params,
                                                                     const float *__restrict__ ebuf,
                                                                     float *__restrict__ gbuf) {
    extern __shared__ __align__(16) float wsm[];
    __shared__ float s_part[kWinThreads * kWinRun];
    const int f = fd.f, N = fd.N, F = fd.F, M = fd.M, E = fd.E, Tk = fd.Tk, tlo = fd.tau_lo, nph = f * f;
    const int b = blockIdx.x;
    const int ph = b % nph, k = (b / nph) % M, e = b / (nph * M);
    const int phy = ph / f, phx = ph - phy * f;
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    const float *dpar = cpar + 2 * M + 2 * e;
    const float u0 = 0.5f * (float)(F - 1);
    const int wx = (int)floorf(u0 + (float)f * (cpar[2 * k] + dpar[0])) - kWinLo;
    const int wy = (int)floorf(u0 + (float)f * (cpar[2 * k + 1] + dpar[1])) - kWinLo;
    // phase-phi positions m with f m + phi in [w, w + kWin) and in the grid
    auto first_m = [&](int w, int p) { int a = w - p; return a >= 0 ? (a + f - 1) / f : -((-a) / f); };
    const int mx0 = max(first_m(wx, phx), 0), my0 = max(first_m(wy, phy), 0);
    const int mx1 = min((wx + kWin - 1 - phx) >= 0 ? (wx + kWin - 1 - phx) / f : -1, N - 1);
    const int my1 = min((wy + kWin - 1 - phy) >= 0 ? (wy + kWin - 1 - phy) / f : -1, N - 1);
    const int nxp = mx1 - mx0 + 1, nyp = my1 - my0 + 1;
    if (nxp <= 0 || nyp <= 0) return;
    // e patch rows [my0 + tlo, my1 + tlo + Tk), cols [mx0 + tlo, mx1 + tlo + Tk)
    const int pw = nxp + Tk - 1, phh = nyp + Tk - 1;
    float *K = wsm, *X = wsm + Tk * Tk;
    const float *kap = fd.kappa + ((long long)e * nph + ph) * Tk * Tk;
    for (int t = threadIdx.x; t < Tk * Tk; t += blockDim.x) K[t] = kap[t];
    const float *ep = ebuf + fd.ebuf_off + (long long)e * N * N;
    for (int t = threadIdx.x; t < phh * pw; t += blockDim.x) {
        const int iy = t / pw, ix = t - iy * pw;
        const int my = my0 + tlo + iy, mx = mx0 + tlo + ix;
        X[t] = (my >= 0 && my < N && mx >= 0 && mx < N) ? ep[(long long)my * N + mx] : 0.f;
    }
    __syncthreads();
    // thread (py, grp): row py of the positions, kernel rows ty = grp mod groups, kWinRun
    // consecutive positions at a time (x values slide through registers: two shared loads per
    // kWinRun multiply-adds); the groups' partials are added in order per position
    const int groups = max(1, min(kWinThreads / nyp, Tk));
    const int py = threadIdx.x % nyp, grp = threadIdx.x / nyp;
    for (int px0 = 0; px0 < nxp; px0 += kWinRun) {
        float acc[kWinRun];
#pragma unroll
        for (int p = 0; p < kWinRun; ++p) acc[p] = 0.f;
        if (grp < groups) {
            for (int ty = grp; ty < Tk; ty += groups) {
                const float *xr = X + (py + ty) * pw + px0, *kr = K + ty * Tk;
                // X rows are pw = nxp + Tk - 1 wide: positions beyond nxp read at most kWinRun - 1
                // values past the row, inside the staged patch or its padding (never used)
                float v[kWinRun];
#pragma unroll
                for (int p = 0; p < kWinRun - 1; ++p) v[p + 1] = xr[p];
                for (int tx = 0; tx < Tk; ++tx) {
#pragma unroll
                    for (int p = 0; p < kWinRun - 1; ++p) v[p] = v[p + 1];
                    v[kWinRun - 1] = xr[tx + kWinRun - 1];
                    const float kv = kr[tx];
#pragma unroll
                    for (int p = 0; p < kWinRun; ++p) acc[p] = fmaf(kv, v[p], acc[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < kWinRun; ++p) s_part[threadIdx.x * kWinRun + p] = acc[p];
        __syncthreads();
        for (int q = threadIdx.x; q < nyp * kWinRun; q += blockDim.x) {
            const int qy = q / kWinRun, p = q - qy * kWinRun, qx = px0 + p;
            if (qx >= nxp) continue;
            float g = 0.f;
            for (int u = 0; u < groups; ++u) g += s_part[(u * nyp + qy) * kWinRun + p];
            gbuf[fd.gbuf_off + ((long long)e * nph + ph) * N * N + (long long)(my0 + qy) * N + (mx0 + qx)] = g;
        }
        __syncthreads();
    }
}

template <int L>
constexpr int bg_smem() {
    return (kBgRows * Bg<L>::RW + L) * (int)sizeof(float2);
}

#define SR_BG_SIZES(X) X(192) X(240) X(288) X(384) X(576) X(768)

template <typename K>
static sr_status bg_open(K kernel, int smem) {
    SR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return SR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
int fft_big_next(int need) {
    static const int sizes[] = {
#define SR_BG_LIST(LL) LL,
        SR_BG_SIZES(SR_BG_LIST)
#undef SR_BG_LIST
    };
    for (int L : sizes)
        if (L >= need) return L;
    return 0;
}

int fft_big_window_smem(int Tk, int f) {
    const int np = kWin / f + 1;
    // the kernel and the patch, and kWinRun floats past the patch that the last row's sliding
    // window reads for positions beyond the row (their sums are never used)
    return (Tk * Tk + (np + Tk - 1) * (np + Tk - 1) + kWinRun) * (int)sizeof(float);
}

sr_status configure_fft_big(int optin) {
    SR_CUDA(pr_fill_dtw());
    sr_status s;
#define SR_BG_CFG(LL)                                                                              \
    if ((s = bg_open(big_load_rows_kernel<LL>, bg_smem<LL>())) != SR_OK) return s;                   \
    if ((s = bg_open(big_cols_kernel<LL, BG_SPLIT>, bg_smem<LL>())) != SR_OK) return s;              \
    if ((s = bg_open(big_cols_kernel<LL, BG_MODEL>, bg_smem<LL>())) != SR_OK) return s;              \
    if ((s = bg_open(big_cols_kernel<LL, BG_ADJ>, bg_smem<LL>())) != SR_OK) return s;                \
    if ((s = bg_open(big_cols_kernel<LL, BG_HJOIN>, bg_smem<LL>())) != SR_OK) return s;              \
    if ((s = bg_open(big_rows_kernel<LL, BG_RESID_ROWS>, bg_smem<LL>())) != SR_OK) return s;         \
    if ((s = bg_open(big_rows_kernel<LL, BG_HOUT_ROWS>, bg_smem<LL>())) != SR_OK) return s;
    SR_BG_SIZES(SR_BG_CFG)
#undef SR_BG_CFG
    SR_CUDA(cudaFuncSetAttribute(big_window_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::min(optin - 2048, 200 * 1024)));
    return SR_OK;
}

static void transpose(const float2 *in, float2 *out, int R, int C, int nimg, cudaStream_t st) {
    dim3 grid((C + 31) / 32, (R + 31) / 32, nimg);
    big_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, out, R, C);
}

template <int L>
static int big_spectra_t(const FieldDev &fd, const float *params, int mode, float2 *zb, float2 *zt, float2 *spec,
                         cudaStream_t st) {
    const int nph = fd.f * fd.f, npr = (nph + 1) / 2, nimg = fd.E * npr;
    const int ny = mode == 0 ? fd.N : fd.Tk;
    big_load_rows_kernel<L><<<dim3((ny + kBgRows - 1) / kBgRows, nimg), kBgThreads, bg_smem<L>(), st>>>(fd, params, mode,
                                                                                                        zb, ny);
    transpose(zb, zt, ny, L, nimg, st);
    BgArgs a{};
    a.zt_in = zt;
    a.spec = spec;
    a.ny = ny;
    a.shift = mode == 1 ? ((fd.tau_lo % L) + L) % L : 0;
    const int H = L / 2 + 1;
    big_cols_kernel<L, BG_SPLIT><<<dim3((H + kBgItems - 1) / kBgItems, nimg), kBgThreads, bg_smem<L>(), st>>>(fd, a);
    return 3;
}

template <int L>
static int big_eval_t(const FieldDev &fd, const float *params, const BigBuffers &bb, float *ebuf, float *gbuf,
                      double *chi_part, double *se_part, cudaStream_t st) {
    int n = big_spectra_t<L>(fd, params, 0, bb.zb, bb.zt, bb.fhat, st);
    const int H = L / 2 + 1, N = fd.N, np = (fd.E + 1) / 2;
    const dim3 cgrid((H + kBgItems - 1) / kBgItems, np), rgrid((N + kBgRows - 1) / kBgRows, np);
    BgArgs a{};
    a.zt_out = bb.zt;
    a.khat = fd.fft_khat;
    a.fhat = bb.fhat;
    big_cols_kernel<L, BG_MODEL><<<cgrid, kBgThreads, bg_smem<L>(), st>>>(fd, a);
    transpose(bb.zt, bb.zb, L, N, np, st);
    big_rows_kernel<L, BG_RESID_ROWS><<<rgrid, kBgThreads, bg_smem<L>(), st>>>(fd, bb.zb, params, ebuf, chi_part,
                                                                              se_part, nullptr);
    transpose(bb.zb, bb.zt, N, L, np, st);
    BgArgs b{};
    b.zt_in = bb.zt;
    b.khat = fd.fft_khat;
    b.acc = bb.acc;
    b.ny = N;
    big_cols_kernel<L, BG_ADJ><<<cgrid, kBgThreads, bg_smem<L>(), st>>>(fd, b);
    n += 5;
    if (fd.M > 0) {
        const int nph = fd.f * fd.f;
        big_window_adj_kernel<<<fd.E * fd.M * nph, kWinThreads, fft_big_window_smem(fd.Tk, fd.f), st>>>(fd, params, ebuf,
                                                                                                      gbuf);
        ++n;
    }
    return n;
}

template <int L>
static int big_hgrad_t(const FieldDev &fd, const BigBuffers &bb, float *grad, cudaStream_t st) {
    const int H = L / 2 + 1, N = fd.N, nph = fd.f * fd.f, npr = (nph + 1) / 2;
    BgArgs a{};
    a.zt_out = bb.zt;
    a.acc = bb.acc;
    a.npairs = (fd.E + 1) / 2;
    big_cols_kernel<L, BG_HJOIN><<<dim3((H + kBgItems - 1) / kBgItems, npr), kBgThreads, bg_smem<L>(), st>>>(fd, a);
    transpose(bb.zt, bb.zb, L, N, npr, st);
    big_rows_kernel<L, BG_HOUT_ROWS><<<dim3((N + kBgRows - 1) / kBgRows, npr), kBgThreads, bg_smem<L>(), st>>>(
        fd, bb.zb, nullptr, nullptr, nullptr, nullptr, grad);
    return 3;
}

int launch_big_kappa(const FieldDev &fd, float2 *zb, float2 *zt, cudaStream_t st) {
    switch (fd.fft_L) {
#define SR_BG_K(LL) \
    case LL:        \
        return big_spectra_t<LL>(fd, nullptr, 1, zb, zt, const_cast<float2 *>(fd.fft_khat), st);
        SR_BG_SIZES(SR_BG_K)
#undef SR_BG_K
        default:
            return 0;
    }
}

int launch_big_eval(const FieldDev &fd, const float *params, const BigBuffers &bb, float *ebuf, float *gbuf,
                    double *chi_part, double *se_part, cudaStream_t st) {
    switch (fd.fft_L) {
#define SR_BG_E(LL) \
    case LL:        \
        return big_eval_t<LL>(fd, params, bb, ebuf, gbuf, chi_part, se_part, st);
        SR_BG_SIZES(SR_BG_E)
#undef SR_BG_E
        default:
            return 0;
    }
}

int launch_big_hgrad(const FieldDev &fd, const BigBuffers &bb, float *grad, cudaStream_t st) {
    switch (fd.fft_L) {
#define SR_BG_H(LL) \
    case LL:        \
        return big_hgrad_t<LL>(fd, bb, grad, st);
        SR_BG_SIZES(SR_BG_H)
#undef SR_BG_H
        default:
            return 0;
    }
}

}  // namespace sr
