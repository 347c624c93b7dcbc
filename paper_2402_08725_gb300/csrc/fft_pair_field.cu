// Per-PSF and per-field transforms of the frequency-domain form (sm_103a): the spectra of the
// folded PSF kernels (at set_psfs), the spectra of the phase images of h (once per evaluation and
// field) and the transform back of the accumulated adjoint spectra (dL/dh).  Each block transforms
// two phases at once as one complex image (fft_pair.cuh).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"
#include "fft_pair.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

// --- per-PSF and per-field transforms (two phases per block) ---------------------------------
// Half spectra of the pair in Z: X_a at out_a, X_b at out_b (if any), rows of pitch HP with the pad
// column zero; each value times W_L^((ky + kx) sh) (sh = 0: no shift).
// The two half spectra of a pair transform Z = X_a + i X_b, in global layout [L][HP]:
//   X_a(k) = (Z(k) + conj Z(-k)) / 2,  X_b(k) = (Z(k) - conj Z(-k)) / (2i),
// each times W_L^((ky + kx) sh) when sh != 0 (the shift theorem); out_b may be null.  A thread
// keeps one column kx (its physical columns and W_L^(kx sh) index) and walks the rows; the
// twiddle of (ky + kx) sh mod L is read from the table, its index kept by additions.
template <int L>
__device__ void split_store(const float2 *Z, float2 *out_a, float2 *out_b, int sh, const float2 *tw) {
    using G = Pr<L>;
    constexpr int H = G::H, HP = G::HP, P = G::P;
    const int rows = blockDim.x / HP;  // rows in parallel
    const int kx = threadIdx.x % HP, ty = threadIdx.x / HP;
    if (ty >= rows) return;
    const bool live = kx < H;
    const int cx = live ? kcol<L>(kx) : 0, cxm = live ? kcol<L>(neg_mod(kx, L)) : 0;
    const int wx = (int)(((long long)kx * sh) % L);
    const int wstep = (int)(((long long)rows * sh) % L);
    int wi = (int)(((long long)ty * sh) % L) + wx;
    if (wi >= L) wi -= L;
    for (int ky = ty; ky < L; ky += rows) {
        float2 xa = make_float2(0.f, 0.f), xb = make_float2(0.f, 0.f);
        if (live) {
            const float2 A = Z[krow<L>(ky) * P + cx];
            const float2 B = Z[krow<L>(neg_mod(ky, L)) * P + cxm];
            xa = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
            xb = make_float2(0.5f * (A.y + B.y), 0.5f * (B.x - A.x));
            if (sh) {
                const float2 w = tw[wi];
                xa = cmul(xa, w);
                xb = cmul(xb, w);
            }
        }
        out_a[ky * HP + kx] = xa;
        if (out_b) out_b[ky * HP + kx] = xb;
        wi += wstep;
        if (wi >= L) wi -= L;
    }
}

// The forward transform along y of a pair whose rows y >= ylim are zero, with ylim <= L/2
// (NZ = 8) or <= L/4 (NZ = 4) and R1 = 16: pass A's 16-point DFTs see non-zero inputs only at
// n1 < NZ, so their first radix-4 stage reduces to one (NZ = 4) or two (NZ = 8) terms; pass B is
// that of cols_fwd.  Same values as cols_fwd (the dropped terms are exact zeros).
template <int L, int NZ>
__device__ __noinline__ void cols_fwd_lead(float2 *Z, int ylim, const float2 *TWL) {
    using G = Pr<L>;
    constexpr int R1 = G::R1, R2 = G::R2, P = G::P;
    static_assert(R1 == 16 && (NZ == 4 || NZ == 8), "pruned column pass: R1 = 16, NZ = 4 or 8");
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < R2 * L; t += nt) {
        const int p = t % L, n2 = t / L;
        float2 *z = Z + pcol<L>(p) + n2 * P;
        float2 v[NZ];
#pragma unroll
        for (int n1 = 0; n1 < NZ; ++n1) v[n1] = n2 + R2 * n1 < ylim ? z[R2 * n1 * P] : make_float2(0.f, 0.f);
        // 16 = 4 x 4: first stage over m1 of v[4 m1 + m2] (only m1 < NZ / 4 non-zero), twiddles
        // W_16^(m2 k1), then 4-point DFTs over m2; X[k1 + 4 k2] is output k1 + 4 k2 of the 16
        float2 a[16];
#pragma unroll
        for (int m2 = 0; m2 < 4; ++m2) {
            float2 q[4];
            if (NZ == 4) {
                q[0] = q[1] = q[2] = q[3] = v[m2];
            } else {
                const float2 t0 = v[m2], t1 = v[4 + m2];
                const float2 t1i = make_float2(t1.y, -t1.x);  // -i t1 (forward W_4)
                q[0] = cadd(t0, t1);
                q[1] = cadd(t0, t1i);
                q[2] = csub(t0, t1);
                q[3] = csub(t0, t1i);
            }
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[k1 * 4 + m2] = twiddle<16, false>(q[k1], m2 * k1);
        }
        float2 out[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 u[4];
#pragma unroll
            for (int m2 = 0; m2 < 4; ++m2) u[m2] = a[k1 * 4 + m2];
            dft<4, false>(u);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) out[k1 + 4 * k2] = u[k2];
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) z[R2 * k1 * P] = k1 == 0 ? out[0] : cmul(out[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < R1 * L; t += nt) {
        const int p = t % L, k1 = t / L;
        float2 *z = Z + pcol<L>(p) + R2 * k1 * P;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = z[n2 * P];
        dft<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) z[k2 * P] = v[k2];
    }
    __syncthreads();
}

// Spectra of the folded PSF kernels (at set_psfs): item = epoch * n_pairs + pair of phases.  The
// phase kernel kappa_phi (Tk x Tk, taps tau_lo .. tau_lo + Tk - 1 on each axis, Tk <= L) belongs on
// the L x L circle with tap tau at tau mod L.  It is placed instead at tau - tau_lo, so that the
// row passes touch only its Tk rows, and the shift is restored on the spectrum (shift theorem):
//   Khat[ky][kx] = W_L^((ky + kx) tau_lo) Khat'[ky][kx],   W_L = exp(-2 pi i / L).
template <int L>
__device__ __noinline__ void kappa_item_pair(const FieldDev &fd, const float *__restrict__ kappa,
                                             float2 *__restrict__ khat, int item) {
    using G = Pr<L>;
    constexpr int P = G::P, HP = G::HP;
    float2 *Z = pr_dyn, *TWL = Z + G::ZN;
    load_twl<L>(TWL, fd.fft_tw);
    const int nph = fd.f * fd.f, npr = (nph + 1) / 2;
    const int i = item / npr, q = item - i * npr;
    const int pa = 2 * q, pb = 2 * q + 1;
    const int Tk = fd.Tk;
    const float *ka = kappa + ((long long)i * nph + pa) * Tk * Tk;
    const float *kb = pb < nph ? ka + Tk * Tk : nullptr;
    for (int t = threadIdx.x; t < Tk * Tk; t += blockDim.x) {
        const int y = t / Tk, x = t - y * Tk;
        Z[y * P + pcol<L>(x)] = make_float2(ka[t], kb ? kb[t] : 0.f);
    }
    __syncthreads();
    rows_fwd<L>(Z, 1, Tk, Tk, TWL);
    if constexpr (Pr<L>::R1 == 16) {
        if (4 * Tk <= L) cols_fwd_lead<L, 4>(Z, Tk, TWL);
        else if (2 * Tk <= L) cols_fwd_lead<L, 8>(Z, Tk, TWL);
        else cols_fwd<L>(Z, 1, Tk, TWL);
    } else {
        cols_fwd<L>(Z, 1, Tk, TWL);
    }
    const int sh = ((fd.tau_lo % L) + L) % L;  // tau_lo mod L
    float2 *out = khat + ((long long)i * nph + pa) * L * HP;
    split_store<L>(Z, out, kb ? out + L * HP : nullptr, sh, fd.fft_tw);
    __syncthreads();
}

__global__ void __launch_bounds__(kFftThreads, 1)
fft_kappa_pair_kernel(FieldDev fd, const float *__restrict__ kappa, float2 *__restrict__ khat) {
    const int n_items = fd.E * ((fd.f * fd.f + 1) / 2);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        switch (fd.fft_L) {
#define SR_PR_KCASE(LL)                                 \
    case LL:                                            \
        kappa_item_pair<LL>(fd, kappa, khat, item);     \
        break;
            SR_PR_SIZES(SR_PR_KCASE)
#undef SR_PR_KCASE
            default:
                break;  // not reached: transform sizes come from the list
        }
    }
}

// The kernel spectra of many problems in one launch: items[j] = (table entry, epoch * n_pairs +
// pair); every block takes items in turn (the spectra live at each entry's fft_khat).
__global__ void __launch_bounds__(kFftThreads, 1)
fft_kappa_pair_batch_kernel(const FieldDev *__restrict__ fields, const int2 *__restrict__ items, int n_items) {
    for (int j = blockIdx.x; j < n_items; j += gridDim.x) {
        const int2 it = items[j];
        const FieldDev &fd = fields[it.x];
        float2 *khat = const_cast<float2 *>(fd.fft_khat);
        switch (fd.fft_L) {
#define SR_PR_BCASE(LL)                                     \
    case LL:                                                \
        kappa_item_pair<LL>(fd, fd.kappa, khat, it.y);      \
        break;
            SR_PR_SIZES(SR_PR_BCASE)
#undef SR_PR_BCASE
            default:
                break;
        }
    }
}

// Hhat_phi: spectra of the phase images of h, F_phi[m] = h[f m + phi], two phases per block.
template <int L>
__device__ __noinline__ void hhat_pair(const FieldDev &fd, const float *__restrict__ params, float2 *__restrict__ hhat_all,
                                       int q) {
    using G = Pr<L>;
    constexpr int P = G::P, HP = G::HP;
    float2 *Z = pr_dyn, *TWL = Z + G::ZN;
    load_twl<L>(TWL, fd.fft_tw);
    const int f = fd.f, N = fd.N, F = fd.F, nph = f * f;
    const int pa = 2 * q, pb = 2 * q + 1;
    const bool hasb = pb < nph;
    const int pay = pa / f, pax = pa - pay * f, pby = pb / f, pbx = pb - pby * f;
    const float *h = params + fd.param_off;
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        const int y = t / N, x = t - y * N;
        const float va = h[(long long)(f * y + pay) * F + f * x + pax];
        const float vb = hasb ? h[(long long)(f * y + pby) * F + f * x + pbx] : 0.f;
        Z[y * P + pcol<L>(x)] = make_float2(va, vb);
    }
    __syncthreads();
    rows_fwd<L>(Z, 1, N, N, TWL);
    cols_fwd<L>(Z, 1, N, TWL);
    float2 *out = hhat_all + fd.fft_hhat_off + (long long)pa * L * HP;
    split_store<L>(Z, out, hasb ? out + L * HP : nullptr, 0, fd.fft_tw);
}

// dL/dh for the transform fields: the chunk accumulators of two phases summed in a fixed order,
// joined as Z = A_a + i A_b on the whole plane (Hermitian extension of each half spectrum),
// transformed back, plus the prior's gradient.
// The sum over a field's work items of their adjoint accumulators at one spectral point, in a
// fixed order shared by acc_reduce and hgrad_pair: 16 interleaved partial sums (item c into
// c mod 16, each in increasing c), combined as a fixed binary tree.
constexpr int kAccParts = 16;

__device__ __forceinline__ float2 acc_tree(const float2 *q) {  // q[0..3] of one group of four parts
    return cadd(cadd(q[0], q[1]), cadd(q[2], q[3]));
}

// Parts 4t .. 4t+3 of the sum at one point (t = 0..3), over items c = u, u + 16, ...
__device__ __forceinline__ float2 acc_group(const float2 *__restrict__ ac, long long cs, int n_chunks, int t) {
    float2 q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = make_float2(0.f, 0.f);
    for (int c = 4 * t; c < n_chunks; c += kAccParts) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (c + v < n_chunks) q[v] = cadd(q[v], __ldg(&ac[(c + v) * cs]));
    }
    return acc_tree(q);
}

// The whole sum at one point by one thread: the 16 parts advanced together (16 loads in flight),
// each in increasing c as in acc_group, then the same trees.
__device__ __forceinline__ float2 acc_sum(const float2 *__restrict__ ac, long long cs, int n_chunks) {
    float2 q[kAccParts];
#pragma unroll
    for (int u = 0; u < kAccParts; ++u) q[u] = make_float2(0.f, 0.f);
    for (int c = 0; c < n_chunks; c += kAccParts) {
#pragma unroll
        for (int u = 0; u < kAccParts; ++u)
            if (c + u < n_chunks) q[u] = cadd(q[u], __ldg(&ac[(c + u) * cs]));
    }
    float2 g[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) g[t] = acc_tree(q + 4 * t);
    return acc_tree(g);
}

// Four threads per spectral point p (phase, row ky, column kx < H), lanes 4i .. 4i+3 of a warp:
// thread t sums parts 4t .. 4t+3, the tree over the four groups is taken by shuffles, and the
// point's sum is written over the first item's accumulator.  Many short chains instead of one
// thread walking every item, so that fields with many items are summed by many blocks.
template <int L>
__device__ __forceinline__ void acc_reduce(const FieldDev &fd, float2 *__restrict__ acc_all, int p, int t) {
    using G = Pr<L>;
    constexpr int H = G::H, HP = G::HP, LHP = L * HP;
    const int nph = fd.f * fd.f;
    const bool live = p < nph * L * H;
    const int pp = live ? p : 0;
    const int ph = pp / (L * H), r = pp - ph * (L * H), ky = r / H, kx = r - ky * H;
    const long long cs = (long long)nph * LHP;
    float2 *ac = acc_all + fd.fft_acc_off + (long long)ph * LHP + ky * HP + kx;
    float2 g = live ? acc_group(ac, cs, fd.fft_n_chunks, t) : make_float2(0.f, 0.f);
    // (g0 + g1) + (g2 + g3) across the four lanes of the point
    float2 o;
    o.x = __shfl_down_sync(0xffffffffu, g.x, 1, 4);
    o.y = __shfl_down_sync(0xffffffffu, g.y, 1, 4);
    g = cadd(g, o);
    o.x = __shfl_down_sync(0xffffffffu, g.x, 2, 4);
    o.y = __shfl_down_sync(0xffffffffu, g.y, 2, 4);
    g = cadd(g, o);
    if (live && t == 0) ac[0] = g;
}

// reduced: the items' accumulators were already summed into the first item's (acc_reduce)
template <int L>
__device__ __noinline__ void hgrad_pair(const FieldDev &fd, const float2 *__restrict__ acc_all,
                                        float *__restrict__ grad, int q, bool reduced) {
    using G = Pr<L>;
    constexpr int P = G::P, H = G::H, HP = G::HP, LHP = L * HP;
    float2 *Z = pr_dyn, *TWL = Z + G::ZN;
    load_twl<L>(TWL, fd.fft_tw);
    const int f = fd.f, N = fd.N, F = fd.F, nph = f * f;
    const int pa = 2 * q, pb = 2 * q + 1;
    const bool hasb = pb < nph;
    const int n_chunks = reduced ? 1 : fd.fft_n_chunks;
    const long long cs = (long long)nph * LHP;
    const float2 *base = acc_all + fd.fft_acc_off;
    for (int idx = threadIdx.x; idx < L * H; idx += blockDim.x) {
        const int ky = idx / H, kx = idx - ky * H;
        const bool selfcol = kx == 0 || 2 * kx == L;
        if (selfcol && 2 * ky > L) continue;  // written by the partner at -ky
        float2 s[2];
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            s[w] = make_float2(0.f, 0.f);
            if (w == 1 && !hasb) continue;
            // the items' sum in acc_reduce's order (a single item: its accumulator as it is)
            const float2 *ac = base + (long long)(w ? pb : pa) * LHP + ky * HP + kx;
            s[w] = n_chunks == 1 ? __ldg(ac) : acc_sum(ac, cs, n_chunks);
        }
        const float2 A = s[0], B = s[1];
        const int r = krow<L>(ky), cx = kcol<L>(kx);
        if (selfcol && (ky == 0 || 2 * ky == L)) {
            Z[r * P + cx] = make_float2(A.x, B.x);
        } else {
            Z[r * P + cx] = make_float2(A.x - B.y, A.y + B.x);                                          // A + i B
            Z[krow<L>(neg_mod(ky, L)) * P + kcol<L>(neg_mod(kx, L))] = make_float2(A.x + B.y, B.x - A.y);  // conj
        }
    }
    __syncthreads();
    cols_inv<L>(Z, 1, N, TWL);
    rows_inv<L>(Z, 1, N, N, TWL);
    const float scale = 1.f / ((float)L * (float)L);
    const int pay = pa / f, pax = pa - pay * f, pby = pb / f, pbx = pb - pby * f;
    const float *T0 = fd.starlet + (long long)fd.J * F * F;
    float *gh = grad + fd.param_off;
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        const int y = t / N, x = t - y * N;
        const float2 v = Z[y * P + pcol<L>(x)];
        const long long ua = (long long)(f * y + pay) * F + f * x + pax;
        gh[ua] = v.x * scale + T0[ua];
        if (hasb) {
            const long long ub = (long long)(f * y + pby) * F + f * x + pbx;
            gh[ub] = v.y * scale + T0[ub];
        }
    }
}

// One block per (transform field, pair of phases): blockIdx.y indexes fft_fields[] (costliest
// fields first), blockIdx.x the pair.
__global__ void __launch_bounds__(kFftThreads, 1)
fft_hhat_pair_kernel(const FieldDev *__restrict__ fields, const int *__restrict__ fft_fields,
                     const float *__restrict__ params, float2 *__restrict__ hhat_all) {
    const FieldDev &fd = fields[fft_fields[blockIdx.y]];
    const int q = blockIdx.x;
    if (2 * q >= fd.f * fd.f) return;
    switch (fd.fft_L) {
#define SR_PR_HCASE(LL)                              \
    case LL:                                         \
        hhat_pair<LL>(fd, params, hhat_all, q);      \
        break;
        SR_PR_SIZES(SR_PR_HCASE)
#undef SR_PR_HCASE
        default:
            break;
    }
}

__global__ void __launch_bounds__(256)
fft_acc_reduce_kernel(const FieldDev *__restrict__ fields, const int *__restrict__ fft_fields,
                      float2 *__restrict__ acc_all) {
    const FieldDev &fd = fields[fft_fields[blockIdx.y]];
    if (fd.fft_n_chunks <= 1) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = g >> 2, t = g & 3;  // four lanes per point
    switch (fd.fft_L) {
#define SR_PR_RCASE(LL)                     \
    case LL:                                \
        acc_reduce<LL>(fd, acc_all, p, t);  \
        break;
        SR_PR_SIZES(SR_PR_RCASE)
#undef SR_PR_RCASE
        default:
            break;
    }
}

__global__ void __launch_bounds__(kFftThreads, 1)
fft_hgrad_pair_kernel(const FieldDev *__restrict__ fields, const int *__restrict__ fft_fields,
                      const float2 *__restrict__ acc_all, float *__restrict__ grad, int reduced) {
    const FieldDev &fd = fields[fft_fields[blockIdx.y]];
    const int q = blockIdx.x;
    if (2 * q >= fd.f * fd.f) return;
    switch (fd.fft_L) {
#define SR_PR_GCASE(LL)                                      \
    case LL:                                                 \
        hgrad_pair<LL>(fd, acc_all, grad, q, reduced != 0);  \
        break;
        SR_PR_SIZES(SR_PR_GCASE)
#undef SR_PR_GCASE
        default:
            break;
    }
}

}  // namespace

template <typename K>
static sr_status open_smem(K kernel, int optin, int *limit) {
    cudaFuncAttributes a;
    SR_CUDA(cudaFuncGetAttributes(&a, kernel));
    const int dyn = optin - (int)a.sharedSizeBytes;
    SR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    *limit = std::min(*limit, dyn);
    return SR_OK;
}

// Opens the largest dynamic shared memory of the per-field kernels; *field_limit is the smallest.
sr_status configure_fft_pair_field(int optin, int *field_limit) {
    SR_CUDA(pr_fill_dtw());
    *field_limit = optin;
    sr_status s;
    if ((s = open_smem(fft_kappa_pair_kernel, optin, field_limit)) != SR_OK) return s;
    if ((s = open_smem(fft_kappa_pair_batch_kernel, optin, field_limit)) != SR_OK) return s;
    if ((s = open_smem(fft_hhat_pair_kernel, optin, field_limit)) != SR_OK) return s;
    if ((s = open_smem(fft_hgrad_pair_kernel, optin, field_limit)) != SR_OK) return s;
    return SR_OK;
}

// Block size of the kernel-spectra launches: of 512, 256 and 128 threads, the one with the most
// threads resident per SM at this shared-memory size, ties to the smaller block (independent blocks
// cover each other's barriers between the passes).  Every output of an item is computed the same
// way whatever the block size, so the spectra do not depend on it.
template <typename K>
static void kappa_block(K kernel, int smem, int *threads, int *occ) {
    *threads = kFftThreads;
    *occ = 1;
    int best = 0;
    for (int t : {kFftThreads, kFftThreads / 2, kFftThreads / 4}) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, t, smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (o >= 1 && o * t >= best) {
            best = o * t;
            *threads = t;
            *occ = o;
        }
    }
}

sr_status launch_fft_kappa_pair_batch(const FieldDev *fields, const int2 *items, int n_items, int L, int n_sms,
                                      cudaStream_t st) {
    if (n_items <= 0) return SR_OK;
    const int smem = fft_pair_field_smem(L);
    int threads = 0, occ = 0;
    kappa_block(fft_kappa_pair_batch_kernel, smem, &threads, &occ);
    const int grid = std::min(n_items, occ * n_sms);
    fft_kappa_pair_batch_kernel<<<grid, threads, smem, st>>>(fields, items, n_items);
    return SR_OK;
}

void launch_fft_kappa_pair(const FieldDev &fd, const float *kappa, float2 *khat, cudaStream_t st) {
    const int n_items = fd.E * ((fd.f * fd.f + 1) / 2);
    const int smem = fft_pair_field_smem(fd.fft_L);
    int threads = 0, occ = 0;
    kappa_block(fft_kappa_pair_kernel, smem, &threads, &occ);
    fft_kappa_pair_kernel<<<n_items, threads, smem, st>>>(fd, kappa, khat);
}

void launch_fft_hhat_pair(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_pairs, int smem,
                          const float *params, float2 *hhat, cudaStream_t st) {
    fft_hhat_pair_kernel<<<dim3(max_pairs, n_fft_fields), kFftThreads, smem, st>>>(fields, fft_fields, params, hhat);
}

int launch_fft_hgrad_pair(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_pairs, int smem,
                          float2 *acc, float *grad, int max_points, int n_sms, cudaStream_t st) {
    // with fewer (field, phase pair) blocks than SMs, the sums over the work items run first on
    // one thread per spectral point; the result is the same either way (same order of the sums)
    const bool reduce = (long long)n_fft_fields * max_pairs < n_sms;
    if (reduce)
        fft_acc_reduce_kernel<<<dim3((4 * max_points + 255) / 256, n_fft_fields), 256, 0, st>>>(fields, fft_fields, acc);
    fft_hgrad_pair_kernel<<<dim3(max_pairs, n_fft_fields), kFftThreads, smem, st>>>(fields, fft_fields, acc, grad,
                                                                                     reduce ? 1 : 0);
    return reduce ? 2 : 1;
}

}  // namespace sr
