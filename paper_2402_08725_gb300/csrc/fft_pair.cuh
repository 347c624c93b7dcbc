// In-place transforms of real image pairs for the frequency-domain form (internal, device code).
//
// Shared by the chunk kernel (fft_pair.cu) and the per-field and per-PSF kernels
// (fft_pair_field.cu); each translation unit holds its own copy of the twiddle table c_dtw and fills
// it in its configure function (pr_fill_dtw).  The layout and the passes are described in
// fft_pair.cu.
#pragma once

#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"
#include "ffsum.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

// --- in-register DFTs -----------------------------------------------------------------------
// W_R^m = exp(-2 pi i m / R), m < R, for the composite sizes 6, 8, 9, 10, 12, 15, 16, 24, 32.
constexpr int kDtwTotal = 6 + 8 + 9 + 10 + 12 + 15 + 16 + 24 + 32;
__constant__ float2 c_dtw[kDtwTotal];
__host__ __device__ constexpr int dtw_off(int R) {
    return R == 6 ? 0 : R == 8 ? 6 : R == 9 ? 14 : R == 10 ? 23 : R == 12 ? 33 : R == 15 ? 45 : R == 16 ? 60
         : R == 24 ? 76 : 100;
}

// v * W_R^m (forward) or v * W_R^-m (inverse), exact for multiples of a quarter turn.
template <int R, bool INV>
__device__ __forceinline__ float2 twiddle(float2 v, int m) {
    if (m == 0) return v;
    if ((4 * m) % R == 0) {
        const int q = (4 * m) / R;  // W^m = (-i)^q
        if (q == 2) return make_float2(-v.x, -v.y);
        const bool minus_i = (q == 1) != INV;
        return minus_i ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    }
    const float2 w = c_dtw[dtw_off(R) + m];
    return INV ? cmulc(v, w) : cmul(v, w);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2 *v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2 *v) {
    const float s1 = INV ? 0.866025403784438647f : -0.866025403784438647f;  // sin(-+2 pi / 3)
    const float2 a = v[0], t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
    v[0] = cadd(a, t);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    const float2 n = make_float2(-s1 * u.y, s1 * u.x);  // i s1 u
    v[1] = cadd(m, n);
    v[2] = csub(m, n);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 *v) {
    const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const float2 c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const float2 di = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);  // +-i d
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, di);
    v[3] = csub(b, di);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2 *v) {
    const float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;  // cos 2pi/5, cos 4pi/5
    const float s1 = INV ? 0.951056516295153572f : -0.951056516295153572f;  // sin(-+2pi/5)
    const float s2 = INV ? 0.587785252292473129f : -0.587785252292473129f;  // sin(-+4pi/5)
    const float2 a = v[0];
    const float2 t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
    const float2 t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
    v[0] = make_float2(a.x + t1.x + t2.x, a.y + t1.y + t2.y);
    const float2 m1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    const float2 m2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    const float2 n1 = make_float2(-(s1 * u1.y + s2 * u2.y), s1 * u1.x + s2 * u2.x);
    const float2 n2 = make_float2(-(s2 * u1.y - s1 * u2.y), s2 * u1.x - s1 * u2.x);
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
}

// 7 points from the symmetric pairs t_j = v_j + v_{7-j}, u_j = v_j - v_{7-j}:
// X_m = v_0 + sum_j cos(2 pi m j / 7) t_j -+ i sum_j sin(2 pi m j / 7) u_j, X_{7-m} with the
// opposite sign of the sine part (m = 1, 2, 3).
template <bool INV>
__device__ __forceinline__ void dft7(float2 *v) {
    constexpr float c1 = 0.623489801858733530f, c2 = -0.222520933956314404f, c3 = -0.900968867902419126f;
    constexpr float s1 = 0.781831482468029809f, s2 = 0.974927912181823607f, s3 = 0.433883739117558120f;
    const float sg = INV ? 1.f : -1.f;
    const float2 a = v[0];
    const float2 t1 = cadd(v[1], v[6]), u1 = csub(v[1], v[6]);
    const float2 t2 = cadd(v[2], v[5]), u2 = csub(v[2], v[5]);
    const float2 t3 = cadd(v[3], v[4]), u3 = csub(v[3], v[4]);
    v[0] = make_float2(a.x + t1.x + t2.x + t3.x, a.y + t1.y + t2.y + t3.y);
    const float C[3][3] = {{c1, c2, c3}, {c2, c3, c1}, {c3, c1, c2}};      // cos(2 pi m j / 7)
    const float S[3][3] = {{s1, s2, s3}, {s2, -s3, -s1}, {s3, -s1, s2}};   // sin(2 pi m j / 7)
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const float *cm = C[m - 1], *sm = S[m - 1];
        const float2 re = make_float2(a.x + cm[0] * t1.x + cm[1] * t2.x + cm[2] * t3.x,
                                      a.y + cm[0] * t1.y + cm[1] * t2.y + cm[2] * t3.y);
        const float2 im = make_float2(sm[0] * u1.x + sm[1] * u2.x + sm[2] * u3.x,
                                      sm[0] * u1.y + sm[1] * u2.y + sm[2] * u3.y);
        const float2 n = make_float2(-sg * im.y, sg * im.x);  // sg i im
        v[m] = cadd(re, n);
        v[7 - m] = csub(re, n);
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *v);

// R = P Q: P-point DFTs of v[Q n1 + n2] over n1, twiddles W_R^(n2 k1), Q-point DFTs over n2;
// X[k1 + P k2] lands in v.
template <int P, int Q, bool INV>
__device__ __forceinline__ void dft_pq(float2 *v) {
    constexpr int R = P * Q;
    float2 a[R];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        float2 t[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) t[n1] = v[Q * n1 + n2];
        dft<P, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) a[k1 * Q + n2] = twiddle<R, INV>(t[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        float2 t[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) t[n2] = a[k1 * Q + n2];
        dft<Q, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *v) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else if constexpr (R == 5) dft5<INV>(v);
    else if constexpr (R == 6) dft_pq<2, 3, INV>(v);
    else if constexpr (R == 7) dft7<INV>(v);
    else if constexpr (R == 8) dft_pq<2, 4, INV>(v);
    else if constexpr (R == 9) dft_pq<3, 3, INV>(v);
    else if constexpr (R == 10) dft_pq<2, 5, INV>(v);
    else if constexpr (R == 12) dft_pq<4, 3, INV>(v);
    else if constexpr (R == 15) dft_pq<3, 5, INV>(v);
    else if constexpr (R == 16) dft_pq<4, 4, INV>(v);
    else if constexpr (R == 24) dft_pq<8, 3, INV>(v);
    else if constexpr (R == 32) dft_pq<8, 4, INV>(v);
    else static_assert(R == 2, "unsupported in-register DFT size");
}

// --- transform geometry -----------------------------------------------------------------------
// L = R1 R2 for the listed sizes (R2 odd where the size allows).
__host__ __device__ constexpr int pr_r1(int L) {
    return L == 24 ? 8 : L == 32 ? 8 : L == 40 ? 8 : L == 48 ? 16 : L == 56 ? 8 : L == 64 ? 16 : L == 72 ? 8 : L == 80 ? 16 : L == 96 ? 16
         : L == 112 ? 16 : L == 128 ? 16 : L == 144 ? 16 : 0;
}
// extra float2 per row beyond R1 S: the row pitch is brought to R2 (mod 16), except at L = 80,
// whose four-pair groups fit in shared memory only without it
__host__ __device__ constexpr int pr_pad(int L, int RW, int R2) {
    return L == 80 ? 0 : (((R2 - RW) % 16) + 16) % 16;
}

template <int L>
struct Pr {
    static constexpr int R1 = pr_r1(L), R2 = L / R1;
    static constexpr int S = (R2 & 1) ? R2 : R2 + 1;  // physical length of a group of R2 positions
    static constexpr int RW = R1 * S;                  // physical width of a row
    static constexpr int P = RW + pr_pad(L, RW, R2);   // row pitch (float2)
    static constexpr int ZN = (L * P + 1) & ~1;        // float2 per pair array (even: 16-byte aligned)
    static constexpr int H = L / 2 + 1, HP = H + 1;    // half spectrum; global rows padded to HP
    static_assert(R1 > 0 && R1 * R2 == L && L % 4 == 0, "transform size not in the list");
};

// physical column of logical x position p (space: p = x; spectra: p = R2 (kx mod R1) + kx / R1)
template <int L>
__device__ __forceinline__ int pcol(int p) {
    return (p / Pr<L>::R2) * Pr<L>::S + p % Pr<L>::R2;
}
// physical column of frequency kx, physical row of frequency ky
template <int L>
__device__ __forceinline__ int kcol(int kx) {
    return (kx % Pr<L>::R1) * Pr<L>::S + kx / Pr<L>::R1;
}
template <int L>
__device__ __forceinline__ int krow(int ky) {
    return Pr<L>::R2 * (ky % Pr<L>::R1) + ky / Pr<L>::R1;
}
__device__ __forceinline__ int neg_mod(int k, int L) { return k == 0 ? 0 : L - k; }

// floor(r / d) for 0 <= r < 1024 d, d <= 2^20: (r + 0.5) / d is at least 0.5 / d from an integer,
// far more than the rounding error of the float product.
__device__ __forceinline__ int fdivq(int r, float inv_d) { return __float2int_rd(((float)r + 0.5f) * inv_d); }

// --- the passes (np arrays at Z + g ZN; twiddles TWL[k1 R2 + n2] = W_L^(n2 k1)) ------------------
// Forward along x of rows [0, nrows): spatial x < xlim (zero beyond) to spectral order.
template <int L>
__device__ __noinline__ void rows_fwd(float2 *Z, int np, int nrows, int xlim, const float2 *TWL) {
    using G = Pr<L>;
    constexpr int R1 = G::R1, R2 = G::R2, S = G::S, P = G::P, ZN = G::ZN;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = nrows * R2;
    const float inv_per = 1.f / (float)per;
    for (int t = tid; t < np * per; t += nt) {
        const int g = fdivq(t, inv_per), rem = t - g * per;
        const int row = rem / R2, n2 = rem - row * R2;
        float2 *z = Z + g * ZN + row * P + n2;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = n2 + R2 * n1 < xlim ? z[n1 * S] : make_float2(0.f, 0.f);
        dft<R1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) z[k1 * S] = k1 == 0 ? v[0] : cmul(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    const int perb = nrows * R1;
    const float inv_perb = 1.f / (float)perb;
    for (int t = tid; t < np * perb; t += nt) {
        const int g = fdivq(t, inv_perb), rem = t - g * perb;
        const int row = rem / R1, k1 = rem - row * R1;
        float2 *z = Z + g * ZN + row * P + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = z[n2];
        dft<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) z[k2] = v[k2];
    }
    __syncthreads();
}

// Inverse along x of rows [0, nrows): spectral order to spatial x, positions x < xlim written.
template <int L>
__device__ __noinline__ void rows_inv(float2 *Z, int np, int nrows, int xlim, const float2 *TWL) {
    using G = Pr<L>;
    constexpr int R1 = G::R1, R2 = G::R2, S = G::S, P = G::P, ZN = G::ZN;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int perb = nrows * R1;
    const float inv_perb = 1.f / (float)perb;
    for (int t = tid; t < np * perb; t += nt) {
        const int g = fdivq(t, inv_perb), rem = t - g * perb;
        const int row = rem / R1, k1 = rem - row * R1;
        float2 *z = Z + g * ZN + row * P + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = z[k2];
        dft<R2, true>(v);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) z[n2] = n2 == 0 ? v[0] : cmulc(v[n2], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    const int per = nrows * R2;
    const float inv_per = 1.f / (float)per;
    for (int t = tid; t < np * per; t += nt) {
        const int g = fdivq(t, inv_per), rem = t - g * per;
        const int row = rem / R2, n2 = rem - row * R2;
        float2 *z = Z + g * ZN + row * P + n2;
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

// Forward along y of every column: spatial rows y < ylim (zero beyond) to spectral order.
template <int L>
__device__ __noinline__ void cols_fwd(float2 *Z, int np, int ylim, const float2 *TWL) {
    using G = Pr<L>;
    constexpr int R1 = G::R1, R2 = G::R2, P = G::P, ZN = G::ZN;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < np * R2 * L; t += nt) {
        const int p = t % L, r = t / L;
        const int n2 = r % R2, g = r / R2;
        float2 *z = Z + g * ZN + pcol<L>(p) + n2 * P;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = n2 + R2 * n1 < ylim ? z[R2 * n1 * P] : make_float2(0.f, 0.f);
        dft<R1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) z[R2 * k1 * P] = k1 == 0 ? v[0] : cmul(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < np * R1 * L; t += nt) {
        const int p = t % L, r = t / L;
        const int k1 = r % R1, g = r / R1;
        float2 *z = Z + g * ZN + pcol<L>(p) + R2 * k1 * P;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = z[n2 * P];
        dft<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) z[k2 * P] = v[k2];
    }
    __syncthreads();
}

// Inverse along y of every column: spectral order to spatial rows, rows y < ylim written.
template <int L>
__device__ __noinline__ void cols_inv(float2 *Z, int np, int ylim, const float2 *TWL) {
    using G = Pr<L>;
    constexpr int R1 = G::R1, R2 = G::R2, P = G::P, ZN = G::ZN;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < np * R1 * L; t += nt) {
        const int p = t % L, r = t / L;
        const int k1 = r % R1, g = r / R1;
        float2 *z = Z + g * ZN + pcol<L>(p) + R2 * k1 * P;
        float2 v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k2] = z[k2 * P];
        dft<R2, true>(v);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) z[n2 * P] = n2 == 0 ? v[0] : cmulc(v[n2], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < np * R2 * L; t += nt) {
        const int p = t % L, r = t / L;
        const int n2 = r % R2, g = r / R2;
        float2 *z = Z + g * ZN + pcol<L>(p) + n2 * P;
        float2 v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = z[R2 * k1 * P];
        dft<R1, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
            if (n2 + R2 * n1 < ylim) z[R2 * n1 * P] = v[n1];
    }
    __syncthreads();
}

template <int L>
__device__ __forceinline__ void load_twl(float2 *TWL, const float2 *tw) {
    constexpr int R2 = Pr<L>::R2;
    for (int n = threadIdx.x; n < L; n += blockDim.x) TWL[n] = tw[(n % R2) * (n / R2)];
}

// --- cache hints --------------------------------------------------------------------------------
// Bulk prefetch of [p, p + bytes) into L2 (a hint; p and bytes multiples of 16, range inside
// one allocation), issued in pieces of at most 64 KB.
__device__ __forceinline__ void prefetch_l2(const void *p, long long bytes) {
    const char *c = static_cast<const char *>(p);
    for (long long off = 0; off < bytes; off += 65536) {
        const unsigned n = (unsigned)((bytes - off) < 65536 ? (bytes - off) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
    }
}

// L2 eviction priorities: a work item's chunk accumulator and the group's kernel spectra stay
// resident across their two uses, while the data and weights and the last reads stream through.
__device__ __forceinline__ unsigned long long l2_policy_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_policy_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// read-only loads (data not written during the kernel)
__device__ __forceinline__ float2 ldg_hint(const float2 *p, unsigned long long pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldg_hint(const float *p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
// The accumulator: volatile, so that its loads and stores keep their program order among
// themselves and against the block barriers; no memory clobber, so that the shared-memory
// accesses and the spectra loads around them can still be scheduled freely (a store's value
// depends on the load of the same element, and different elements never alias).
__device__ __forceinline__ float2 ld_hint(const float2 *p, unsigned long long pol) {
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float2 *p, float2 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol));
}

// Declared here rather than passed down, so that the per-size bodies (not inlined) still address
// them as shared memory.
extern __shared__ __align__(16) float2 pr_dyn[];

#define SR_PR_SIZES(X) X(24) X(32) X(40) X(48) X(56) X(64) X(72) X(80) X(96) X(112) X(128) X(144)

// Fills this translation unit's twiddle table.
inline cudaError_t pr_fill_dtw() {
    float2 tw[kDtwTotal];
    for (int R : {6, 8, 9, 10, 12, 15, 16, 24, 32})
        for (int m = 0; m < R; ++m) {
            const double a = -2.0 * M_PI * (double)m / (double)R;
            tw[dtw_off(R) + m] = make_float2((float)cos(a), (float)sin(a));
        }
    return cudaMemcpyToSymbol(c_dtw, tw, sizeof(tw));
}

}  // namespace
}  // namespace sr
