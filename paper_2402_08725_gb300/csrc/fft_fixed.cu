// Frequency-domain chunk kernel for transform sizes known at compile time (sm_103a).
//
// Computes per epoch exactly what the frequency-domain form defines (fft.cu): the model spectrum
// sum_phi Khat_phi (Hhat_phi + Phat_phi), its inverse real transform, the weighted residual and
// chi^2, the forward transform of e, the adjoint spectra conj(Khat_phi) ehat accumulated per chunk,
// and the point sources' Parseval products.  What differs is how the transforms run:
//
//  * L = R1 R2 is a template parameter taken from a fixed list (multiples of 4, 16..144).  A
//    length-L transform is two passes of in-register DFTs: R2 threads per transform each take
//    an R1-point DFT of the elements n2 + R2 n1 and multiply by W_L^(n2 k1); then R1 threads
//    each take an R2-point DFT of the results k1 and write X[k1 + R1 k2].  A real L x L image
//    is transformed as row pairs (two real rows in one complex row), split into the half
//    spectrum, then columns, so one 2-D transform is four passes with a barrier after each.
//  * G epochs of a chunk run side by side (G = 1, 2 or 4, chosen on the host so that their
//    buffers fit in shared memory; G > 1 only for fields with at most one point source): small
//    transforms fill the block, and the chunk accumulator is read and written once per group
//    instead of once per epoch.
//  * the spectral loops take 4 (point, epoch) pairs per thread per batch, so that their global
//    loads (kernel spectra, h spectra, accumulator) are in flight together; L2 eviction
//    priorities keep the chunk accumulator and the epoch's kernel spectra resident.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "cplx.cuh"
#include "ffsum.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

// --- in-register DFTs -----------------------------------------------------------------------
// W_R^m = exp(-2 pi i m / R), m < R, for the composite sizes 6, 8, 9, 10, 12, 16.
constexpr int kDtwTotal = 61;
__constant__ float2 c_dtw[kDtwTotal];
__host__ __device__ constexpr int dtw_off(int R) { return R == 6 ? 0 : R == 8 ? 6 : R == 9 ? 14 : R == 10 ? 23 : R == 12 ? 33 : 45; }

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
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else if constexpr (R == 5) dft5<INV>(v);
    else if constexpr (R == 6) dft_pq<2, 3, INV>(v);
    else if constexpr (R == 8) dft_pq<2, 4, INV>(v);
    else if constexpr (R == 9) dft_pq<3, 3, INV>(v);
    else if constexpr (R == 10) dft_pq<2, 5, INV>(v);
    else if constexpr (R == 12) dft_pq<4, 3, INV>(v);
    else if constexpr (R == 16) dft_pq<4, 4, INV>(v);
    else static_assert(R == 2, "unsupported in-register DFT size");
}

// --- transform geometry -----------------------------------------------------------------------
__host__ __device__ constexpr int fx_r1(int L) {
    return L == 16 ? 4 : L == 20 ? 5 : L == 24 ? 6 : L == 32 ? 8 : L == 36 ? 6 : L == 40 ? 8 : L == 48 ? 8
         : L == 60 ? 10 : L == 64 ? 8 : L == 72 ? 9 : L == 80 ? 10 : L == 96 ? 12 : L == 100 ? 10
         : L == 108 ? 12 : L == 120 ? 12 : L == 128 ? 16 : L == 144 ? 12 : 0;
}

// Buffer layouts (float2 units), per epoch, each of the two buffers:
//   row pairs       p * PX + x                 (p < np, x < L)
//   row pass 1 out  p * PY + k1 * S + n2       (S odd: the R2-point loads of pass 2 are conflict-free)
//   half spectrum   ky * HP + kx               (kx < H = L/2 + 1; HP = H + 1 even, as in global
//                                               memory, so that column pairs are 16-byte aligned)
template <int L>
struct Fx {
    static constexpr int R1 = fx_r1(L), R2 = L / R1, H = L / 2 + 1, LH = L * H;
    static constexpr int HP = H + 1, LHP = L * HP;  // global spectra: row pitch HP (zero pad column)
    static constexpr int S = (R2 & 1) ? R2 : R2 + 1, PX = L, PY = R1 * S;
    // per-buffer float2 count of a full-width transform (L/2 row pairs, every column), even
    static constexpr int EBF0 = (L / 2) * (PY > PX ? PY : PX) > LHP ? (L / 2) * (PY > PX ? PY : PX) : LHP;
    static constexpr int EBF = (EBF0 + 1) & ~1;
    static_assert(R1 > 0 && R1 * R2 == L && L % 4 == 0, "transform size not in the list");
};

// floor(r / d) for 0 <= r < 1024 d and d <= 1024: (r + 0.5) / d is at least 0.5 / d away from an
// integer, far more than the rounding error of the float product.
__device__ __forceinline__ int fdivq(int r, float inv_d) { return __float2int_rd(((float)r + 0.5f) * inv_d); }

// Forward real 2-D transform of G epochs.  A[g]: np row pairs (pitch PX), columns >= N read as
// zero; result: the half spectrum in A[g] (pitch H).  TWL[k1 R2 + n2] = W_L^(n2 k1).
template <int L>
__device__ void fx_fwd2d(float2 *A, float2 *B, int EB, int G, int np, float inv_np, int N, const float2 *TWL) {
    using P = Fx<L>;
    constexpr int R1 = P::R1, R2 = P::R2, H = P::H, HP = P::HP, S = P::S, PX = P::PX, PY = P::PY;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < G * np * R2; t += nt) {  // rows, pass 1
        const int n2 = t % R2, r = t / R2;
        const int g = fdivq(r, inv_np), p = r - g * np;
        const float2 *src = A + g * EB + p * PX;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int x = R2 * n1 + n2;
            v[n1] = x < N ? src[x] : make_float2(0.f, 0.f);
        }
        dft<R1, false>(v);
        float2 *dst = B + g * EB + p * PY + n2;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dst[k1 * S] = k1 == 0 ? v[0] : cmul(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < G * np * R1; t += nt) {  // rows, pass 2
        const int k1 = t % R1, r = t / R1;
        const int g = fdivq(r, inv_np), p = r - g * np;
        const float2 *src = B + g * EB + p * PY + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = src[n2];
        dft<R2, false>(v);
        float2 *dst = A + g * EB + p * PX + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) dst[R1 * k2] = v[k2];
    }
    __syncthreads();
    for (int t = tid; t < G * H * R2; t += nt) {  // split into row spectra, columns pass 1
        const int kx = t % H, r = t / H;
        const int n2 = r % R2, g = r / R2;
        const float2 *src = A + g * EB;
        const int kxm = kx == 0 ? 0 : L - kx;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int y = R2 * n1 + n2;
            float2 o = make_float2(0.f, 0.f);
            if (y < 2 * np) {
                const float2 *row = src + (y >> 1) * PX;
                const float2 a = row[kx], b = conjf2(row[kxm]);
                o = (y & 1) ? make_float2(0.5f * (a.y - b.y), -0.5f * (a.x - b.x))   // (a - b) / (2i)
                            : make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));   // (a + b) / 2
            }
            v[n1] = o;
        }
        dft<R1, false>(v);
        float2 *dst = B + g * EB + n2 * HP + kx;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dst[k1 * R2 * HP] = k1 == 0 ? v[0] : cmul(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < G * H * R1; t += nt) {  // columns, pass 2
        const int kx = t % H, r = t / H;
        const int k1 = r % R1, g = r / R1;
        const float2 *src = B + g * EB + k1 * R2 * HP + kx;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = src[n2 * HP];
        dft<R2, false>(v);
        float2 *dst = A + g * EB + k1 * HP + kx;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) dst[R1 * k2 * HP] = v[k2];
    }
    __syncthreads();
}

// Inverse real 2-D transform of G epochs: the half spectrum in A[g] (pitch H) becomes np row
// pairs of the unscaled image (times L^2) in A[g] (pitch PX), columns < N written.
template <int L>
__device__ void fx_inv2d(float2 *A, float2 *B, int EB, int G, int np, float inv_np, int N, const float2 *TWL) {
    using P = Fx<L>;
    constexpr int R1 = P::R1, R2 = P::R2, H = P::H, HP = P::HP, S = P::S, PX = P::PX, PY = P::PY;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < G * H * R2; t += nt) {  // columns, pass 1
        const int kx = t % H, r = t / H;
        const int n2 = r % R2, g = r / R2;
        const float2 *src = A + g * EB + n2 * HP + kx;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = src[n1 * R2 * HP];
        dft<R1, true>(v);
        float2 *dst = B + g * EB + n2 * HP + kx;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dst[k1 * R2 * HP] = k1 == 0 ? v[0] : cmulc(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < G * H * R1; t += nt) {  // columns, pass 2: rows y < 2 np only
        const int kx = t % H, r = t / H;
        const int k1 = r % R1, g = r / R1;
        const float2 *src = B + g * EB + k1 * R2 * HP + kx;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = src[n2 * HP];
        dft<R2, true>(v);
        float2 *dst = A + g * EB + k1 * HP + kx;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            if (k1 + R1 * k2 < 2 * np) dst[R1 * k2 * HP] = v[k2];
    }
    __syncthreads();
    for (int t = tid; t < G * np * R2; t += nt) {  // merge rows 2p, 2p+1; rows pass 1
        const int n2 = t % R2, r = t / R2;
        const int g = fdivq(r, inv_np), p = r - g * np;
        const float2 *r1 = A + g * EB + (2 * p) * HP, *r2 = r1 + HP;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int x = R2 * n1 + n2;
            if (x < H) {
                const float2 a = r1[x], b = r2[x];
                v[n1] = make_float2(a.x - b.y, a.y + b.x);   // a + i b
            } else {
                const float2 a = r1[L - x], b = r2[L - x];
                v[n1] = make_float2(a.x + b.y, -a.y + b.x);  // conj(a) + i conj(b)
            }
        }
        dft<R1, true>(v);
        float2 *dst = B + g * EB + p * PY + n2;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dst[k1 * S] = k1 == 0 ? v[0] : cmulc(v[k1], TWL[k1 * R2 + n2]);
    }
    __syncthreads();
    for (int t = tid; t < G * np * R1; t += nt) {  // rows, pass 2: columns x < N only
        const int k1 = t % R1, r = t / R1;
        const int g = fdivq(r, inv_np), p = r - g * np;
        const float2 *src = B + g * EB + p * PY + k1 * S;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) v[n2] = src[n2];
        dft<R2, true>(v);
        float2 *dst = A + g * EB + p * PX + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            if (k1 + R1 * k2 < N) dst[R1 * k2] = v[k2];
    }
    __syncthreads();
}

// Bulk prefetch of [p, p + bytes) into L2 (a hint; p and bytes multiples of 16, range inside
// one allocation), issued in pieces of at most 64 KB.
__device__ __forceinline__ void prefetch_l2(const void *p, long long bytes) {
    const char *c = static_cast<const char *>(p);
    for (long long off = 0; off < bytes; off += 65536) {
        const unsigned n = (unsigned)((bytes - off) < 65536 ? (bytes - off) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
    }
}

// L2 eviction priorities.  Per SM a large-L work item keeps its chunk accumulator (f^2 L (L/2+1)
// complex) and the current epoch's kernel spectra live across the epoch, while the data,
// weights and last reads of the spectra stream through: without hints the streamed lines
// evict the accumulator between its read-modify-writes.
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
// two complex values (16 bytes: a column pair of a padded spectrum row)
__device__ __forceinline__ float4 ldg4_hint(const float2 *p, unsigned long long pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
// The accumulator: volatile, so that its loads and stores keep their program order among
// themselves and against the block barriers; no memory clobber, so that the shared-memory reads
// and the spectra loads around them can still be scheduled freely (a store's value depends on the
// load of the same element, and different elements never alias).
__device__ __forceinline__ float2 ld_hint(const float2 *p, unsigned long long pol) {
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float2 *p, float2 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol));
}
__device__ __forceinline__ float4 ld4_hint(const float2 *p, unsigned long long pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st4_hint(float2 *p, float4 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol));
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

constexpr int kBatch = 4;  // (spectral point, epoch) pairs per thread per batch of loads
constexpr int kPairRows = 2;  // rows per step of the one-epoch loops (two columns per row)
constexpr int kMaxG = 4;   // epochs per group (<= kBatch: a batch holds every epoch of its points)
// reduced values per group: G (2 + 3 M) with G > 1 only when M <= 1
constexpr int kRedVals = (kMaxG * 5 > 2 + 3 * kFftMaxSources) ? kMaxG * 5 : 2 + 3 * kFftMaxSources;
static_assert(kMaxG <= kBatch && kFftMaxSources <= kBatch, "accumulators are indexed by batch element");
static_assert(kRedVals <= kFftThreads / 32 && kFftThreads / 32 <= 32, "one warp per reduced value, one lane per warp");

struct FxShared {
    float2 red[kRedVals][kFftThreads / 32];  // compensated partial sums (hi, lo)
    // the work item's parameters: amplitudes a_{i,k}, epoch shifts delta_i, backgrounds gamma_i
    // of its epochs, and the source positions c_k (loaded once per item)
    float ia[kFftChunk * kFftMaxSources];
    float id[2 * kFftChunk];
    float ig[kFftChunk];
    float ic[2 * kFftMaxSources];
    int item;
};
// Declared here rather than passed down, so that the per-size bodies (not inlined) still address
// them as shared memory.
extern __shared__ __align__(16) float2 fx_dyn[];
__shared__ FxShared fx_sh;

// One item (x = field, y = first epoch, z = end, w = chunk index within the field), in groups
// of G epochs.  Not inlined: each size is register-allocated on its own (one call per item).
template <int L>
__device__ __noinline__ void chunk_item_fixed(const FieldDev &fd, const int4 item, const float *__restrict__ params,
                                 const float2 *__restrict__ hhat_all, float2 *__restrict__ acc_all,
                                 double *__restrict__ chi_part, double *__restrict__ se_part,
                                 float *__restrict__ ps_da, float *__restrict__ ps_du) {
    float2 *const fsm = fx_dyn;
    FxShared &sh = fx_sh;
    using P = Fx<L>;
    constexpr int H = P::H, R2 = P::R2, HP = P::HP, LHP = P::LHP;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int f = fd.f, N = fd.N, F = fd.F, M = fd.M, E = fd.E, nph = f * f;
    const int G = fd.fft_G, lgG = G == 4 ? 2 : G == 2 ? 1 : 0;
    const int EB = fd.fft_EB;
    const int np = (N + 1) / 2;
    const float inv_np = 1.f / (float)np;
    float2 *A = fsm, *B = fsm + G * EB, *TWL = B + G * EB, *tw = TWL + L;
    // point-source 1-D spectra per epoch of the group: [G][M][f][H] x-profiles, x-derivatives,
    // then [G][M][f][L] y-profiles, y-derivatives
    const int MfH = M * f * H, MfL = M * f * L;
    float2 *gsx = tw + L, *gsxd = gsx + G * MfH, *gsy = gsxd + G * MfH, *gsyd = gsy + G * MfL;
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    for (int n = tid; n < L; n += nt) {
        tw[n] = fd.fft_tw[n];
        TWL[n] = fd.fft_tw[(n % R2) * (n / R2)];
    }
    {
        const int n_ep = item.z - item.y;
        for (int t = tid; t < n_ep * M; t += nt) sh.ia[t] = hpar[(long long)F * F + (long long)item.y * M + t];
        for (int t = tid; t < 2 * n_ep; t += nt) sh.id[t] = cpar[2 * M + 2 * item.y + t];
        for (int t = tid; t < n_ep; t += nt) sh.ig[t] = cpar[2 * M + 2 * E + item.y + t];
        for (int t = tid; t < 2 * M; t += nt) sh.ic[t] = cpar[t];
    }
    __syncthreads();
    const float2 *hh = hhat_all + fd.fft_hhat_off;
    float2 *acc = acc_all + fd.fft_acc_off + (long long)item.w * nph * LHP;
    const float u0 = 0.5f * (float)(F - 1);
    const float scale = 1.f / ((float)L * (float)L);
    const int nsub = nw >> lgG;  // warps per epoch in the residual
    // spectral loops: thread (ty, tx) takes column tx and rows ty + RP r
    constexpr int RP = kFftThreads / H;
    const int tx = tid % H, ty = tid / H;
    const int rstep = (kBatch >> lgG) * RP;
    const float wgt = (tx == 0 || 2 * tx == L) ? 1.f : 2.f;  // Parseval weight of column tx
    // one-epoch loops: thread (ty2, cp) = (tid / HH, tid mod HH) takes the column pair
    // (c0, c1) = (2 cp, 2 cp + 1) (c1 = H is the zero pad column) of rows ty2 + RP2 r
    constexpr int HH = HP / 2, RP2 = kFftThreads / HH;
    const int cp = tid % HH, ty2 = tid / HH, c0 = 2 * cp, c1 = c0 + 1;
    const bool has1 = c1 < H;
    const float wgt0 = (c0 == 0 || 2 * c0 == L) ? 1.f : 2.f, wgt1 = has1 ? (2 * c1 == L ? 1.f : 2.f) : 0.f;
    const unsigned long long pol_last = l2_policy_last(), pol_first = l2_policy_first();
    const int nv = 2 + 3 * M;    // reduced values per epoch
    for (int i0 = item.y; i0 < item.z; i0 += G) {
        const int Ge = min(G, item.z - i0);
        const float2 *kh = fd.fft_khat + (long long)i0 * nph * LHP;  // [g][phi][L][HP]
        const float *apar = sh.ia + (i0 - item.y) * M;  // a_{i0 + g, k} at g M + k
        // This group's kernel spectra go to L2 while the window spectra are computed, and the
        // next group's data and weights while this one computes (sizes are multiples of 16
        // bytes: L*H is even, and N*N*4 when N is even).  The next group's kernel spectra are not
        // prefetched: with every SM holding a large-L item, one more epoch of spectra per SM
        // overflows L2.
        if (tid == 0) prefetch_l2(kh, (long long)Ge * nph * LHP * (long long)sizeof(float2));
        if (tid == 0 && i0 + G < item.z) {
            const int Gn = min(G, item.z - i0 - G);
            if ((N & 1) == 0) {
                prefetch_l2(fd.d + (long long)(i0 + G) * N * N, (long long)Gn * N * N * 4);
                prefetch_l2(fd.w + (long long)(i0 + G) * N * N, (long long)Gn * N * N * 4);
            }
        }
        // 1-D transforms of the window profiles g1(u - c) and g1(u - c) (u - c) / sigma^2
        {
            const int nx = MfH, ny = MfL, per = nx + ny;
            for (int idx = tid; idx < Ge * per; idx += nt) {
                const int g = idx / per, rr = idx - g * per;
                const bool isx = rr < nx;
                const int r = isx ? rr : rr - nx;
                const int len = isx ? H : L;
                const int kf = r / len, kk = r - kf * len;
                const int k = kf / f, phs = kf - k * f;
                const float cpos = sh.ic[2 * k + (isx ? 0 : 1)], dl = sh.id[2 * (i0 - item.y + g) + (isx ? 0 : 1)];
                const float cc = u0 + (float)f * (cpos + dl);
                const int lo = (int)floorf(cc) - kWinLo;
                int m0 = lo - phs;
                m0 = m0 >= 0 ? (m0 + f - 1) / f : -((-m0) / f);
                float2 v = make_float2(0.f, 0.f), vd = make_float2(0.f, 0.f);
                for (int m = m0;; ++m) {
                    const int u = f * m + phs;
                    if (u >= lo + kWin) break;
                    if (u < 0 || u >= F) continue;
                    const float t = src_offset(u, F, f, cpos, dl);
                    const float gv = kGauss1Norm * exp2f(-t * t);
                    const float gd = gv * t * kGaussInvSig2;
                    const float2 w = tw[(kk * m) % L];  // kk < L, 0 <= m <= N + 1: no overflow
                    v.x += gv * w.x;
                    v.y += gv * w.y;
                    vd.x += gd * w.x;
                    vd.y += gd * w.y;
                }
                if (isx) {
                    gsx[g * MfH + r] = v;
                    gsxd[g * MfH + r] = vd;
                } else {
                    gsy[g * MfL + r] = v;
                    gsyd[g * MfL + r] = vd;
                }
            }
        }
        __syncthreads();
        // model spectra: sum_phi Khat_{g,phi} (Hhat_phi + sum_k a_{g,k} gx gy).  Thread
        // (ty, tx) = (tid / H, tid mod H) takes column kx = tx and rows ty + RP r, so there is no
        // per-point index division; batch element j takes epoch j mod G of row row0 + (j / G) RP
        // One epoch per group (the large transforms): the column pairs of kPairRows rows per step,
        // with 16-byte loads; the sources' column profiles a_k gx_k are loaded once per step.
        if (G == 1 && ty2 < RP2) {
            for (int row0 = ty2; row0 < L; row0 += kPairRows * RP2) {
                float2 m0[kPairRows], m1[kPairRows];
#pragma unroll
                for (int j = 0; j < kPairRows; ++j) m0[j] = m1[j] = make_float2(0.f, 0.f);
                for (int ph = 0; ph < nph; ++ph) {
                    const int phy = ph / f, phx = ph - phy * f;
                    float4 kv[kPairRows], sv[kPairRows];
#pragma unroll
                    for (int j = 0; j < kPairRows; ++j) {
                        const int row = row0 + j * RP2;
                        const int off = row * HP + c0;
                        kv[j] = row < L ? ldg4_hint(kh + ph * LHP + off, pol_last) : make_float4(0.f, 0.f, 0.f, 0.f);
                        sv[j] = row < L ? ldg4_hint(hh + ph * LHP + off, pol_last) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    for (int k = 0; k < M; ++k) {
                        const float a = apar[k];
                        const float2 *gxk = gsx + (k * f + phx) * H;
                        const float2 gx0 = gxk[c0], gx1 = has1 ? gxk[c1] : make_float2(0.f, 0.f);
                        const float2 agx0 = make_float2(a * gx0.x, a * gx0.y), agx1 = make_float2(a * gx1.x, a * gx1.y);
                        const float2 *gy = gsy + (k * f + phy) * L;
#pragma unroll
                        for (int j = 0; j < kPairRows; ++j) {
                            const int row = row0 + j * RP2;
                            if (row < L) {
                                const float2 g = gy[row], p0 = cmul(agx0, g), p1 = cmul(agx1, g);
                                sv[j] = make_float4(sv[j].x + p0.x, sv[j].y + p0.y, sv[j].z + p1.x, sv[j].w + p1.y);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kPairRows; ++j) {
                        m0[j] = cadd(m0[j], cmul(lo2(kv[j]), lo2(sv[j])));
                        m1[j] = cadd(m1[j], cmul(hi2(kv[j]), hi2(sv[j])));
                    }
                }
#pragma unroll
                for (int j = 0; j < kPairRows; ++j) {
                    const int row = row0 + j * RP2;
                    if (row < L) {
                        // one 16-byte store of the pair (the pad column's value is zero)
                        *reinterpret_cast<float4 *>(A + row * HP + c0) = make_float4(m0[j].x, m0[j].y, m1[j].x, m1[j].y);
                    }
                }
            }
        }
        // Several epochs per group (then at most one source): batch element j takes epoch
        // j mod G of row row0 + (j / G) RP.
        if (G > 1 && ty < RP) {
            for (int row0 = ty; row0 < L; row0 += rstep) {
                float2 m[kBatch];
#pragma unroll
                for (int j = 0; j < kBatch; ++j) m[j] = make_float2(0.f, 0.f);
                for (int ph = 0; ph < nph; ++ph) {
                    const int phy = ph / f, phx = ph - phy * f;
                    float2 kv[kBatch], sv[kBatch];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int g = j & (G - 1), row = row0 + (j >> lgG) * RP;
                        const bool ok = row < L && g < Ge;
                        const int off = row * HP + tx;
                        kv[j] = ok ? ldg_hint(kh + (g * nph + ph) * LHP + off, pol_last) : make_float2(0.f, 0.f);
                        sv[j] = ok ? ldg_hint(hh + ph * LHP + off, pol_last) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int g = j & (G - 1), row = row0 + (j >> lgG) * RP;
                        if (row < L && g < Ge) {
                            for (int k = 0; k < M; ++k) {
                                const float2 pr = cmul(gsx[g * MfH + (k * f + phx) * H + tx],
                                                       gsy[g * MfL + (k * f + phy) * L + row]);
                                const float a = apar[g * M + k];
                                sv[j].x += a * pr.x;
                                sv[j].y += a * pr.y;
                            }
                        }
                        m[j] = cadd(m[j], cmul(kv[j], sv[j]));
                    }
                }
#pragma unroll
                for (int j = 0; j < kBatch; ++j) {
                    const int g = j & (G - 1), row = row0 + (j >> lgG) * RP;
                    if (row < L && g < Ge) A[g * EB + row * HP + tx] = m[j];
                }
            }
        }
        __syncthreads();
        fx_inv2d<L>(A, B, EB, Ge, np, inv_np, N, TWL);
        // residual on [0,N)^2 in place (e for the forward transform), chi^2 and sum e: the warps
        // w with w mod G = g take the row pairs of epoch g
        {
            const int g = warp & (G - 1), sub = warp >> lgG;
            FSum chi = fsum_zero(), se = fsum_zero();
            if (g < Ge) {
                const int i = i0 + g;
                const float gam = sh.ig[i - item.y];
                const float bg = (float)(f * f) * gam;
                const float *dd = fd.d + (long long)i * N * N, *ww = fd.w + (long long)i * N * N;
                // two row pairs per iteration, so that 32 data and weight loads per lane are in
                // flight together
                for (int p0 = sub; p0 < np; p0 += 2 * nsub) {
                    float chi_r = 0.f, se_r = 0.f;
                    for (int x0 = 0; x0 < N; x0 += 128) {
                        float dv[2][4][2], wv[2][4][2];
#pragma unroll
                        for (int rp = 0; rp < 2; ++rp) {
                            const int p = p0 + rp * nsub;
#pragma unroll
                            for (int jx = 0; jx < 4; ++jx) {
                                const int x = x0 + 32 * jx + lane;
#pragma unroll
                                for (int q = 0; q < 2; ++q) {
                                    const int y = 2 * p + q;
                                    const bool in = p < np && y < N && x < N;
                                    dv[rp][jx][q] = in ? ldg_hint(dd + y * N + x, pol_first) : 0.f;
                                    wv[rp][jx][q] = in ? ldg_hint(ww + y * N + x, pol_first) : 0.f;
                                }
                            }
                        }
#pragma unroll
                        for (int rp = 0; rp < 2; ++rp) {
                            const int p = p0 + rp * nsub;
                            if (p < np) {
                                float2 *row = A + g * EB + p * P::PX;
#pragma unroll
                                for (int jx = 0; jx < 4; ++jx) {
                                    const int x = x0 + 32 * jx + lane;
                                    if (x < N) {
                                        const float2 mv = row[x];
                                        float e2[2] = {0.f, 0.f};
#pragma unroll
                                        for (int q = 0; q < 2; ++q) {
                                            if (2 * p + q < N) {
                                                const float Mv = (q ? mv.y : mv.x) * scale + bg;
                                                const float res = dv[rp][jx][q] - Mv;
                                                chi_r += 0.5f * wv[rp][jx][q] * res * res;
                                                e2[q] = -wv[rp][jx][q] * res;
                                                se_r += e2[q];
                                            }
                                        }
                                        row[x] = make_float2(e2[0], e2[1]);
                                    }
                                }
                            }
                        }
                    }
                    chi = fsum_add(chi, chi_r);
                    se = fsum_add(se, se_r);
                }
            }
            chi = fsum_warp(chi);
            se = fsum_warp(se);
            if (lane == 0 && g < Ge) {
                sh.red[g * nv + 0][sub] = make_float2(chi.hi, chi.lo);
                sh.red[g * nv + 1][sub] = make_float2(se.hi, se.lo);
            }
        }
        __syncthreads();
        fx_fwd2d<L>(A, B, EB, Ge, np, inv_np, N, TWL);
        // adjoint spectra: acc_phi += sum_g conj(Khat_{g,phi}) ehat_g (epochs in order), and the
        // Parseval products of the sources (weights 1 at kx = 0 and L/2, 2 elsewhere).  With
        // G > 1 (then M <= 1) the products are kept per batch element and folded per epoch
        // below; with G = 1 per source (M <= kFftMaxSources <= kBatch).
        const bool first = i0 == item.y, last = i0 + G >= item.z;
        float pa[kBatch], px[kBatch], py[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) pa[j] = px[j] = py[j] = 0.f;
        // One epoch per group: batch element j is row row0 + j RP.  With the column tx fixed,
        // the Parseval sums factor: sum_rows w Re(G conj(gx gy)) = w Re(conj(gx) U) with
        // U = sum_rows G conj(gy) (and V with the y-derivative profile), so per point only U and V
        // are accumulated and the column profiles are applied once per step.
        // (compiled for at most one source, the common case, and for up to kFftMaxSources)
        auto adj_one_epoch = [&](auto ms_tag) {
            constexpr int MS = decltype(ms_tag)::value;
            for (int row0 = ty2; row0 < L; row0 += kPairRows * RP2) {
                for (int ph = 0; ph < nph; ++ph) {
                    const int phy = ph / f, phx = ph - phy * f;
                    float2 *ap = acc + ph * LHP + c0;
                    float4 kv[kPairRows], av[kPairRows];
#pragma unroll
                    for (int j = 0; j < kPairRows; ++j) {
                        const int row = row0 + j * RP2;
                        kv[j] = row < L ? ldg4_hint(kh + ph * LHP + row * HP + c0, pol_first)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                        av[j] = (row < L && !first) ? ld4_hint(ap + row * HP, pol_last) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    float2 U0[MS], U1[MS], V0[MS], V1[MS];
#pragma unroll
                    for (int k = 0; k < MS; ++k) U0[k] = U1[k] = V0[k] = V1[k] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < kPairRows; ++j) {
                        const int row = row0 + j * RP2;
                        if (row < L) {
                            // one 16-byte load of the pair; the pad slot holds no transform output
                            const float4 e = *reinterpret_cast<const float4 *>(A + row * HP + c0);
                            const float2 e0 = lo2(e), e1 = has1 ? hi2(e) : make_float2(0.f, 0.f);
                            const float2 G0 = cmulc(e0, lo2(kv[j])), G1 = cmulc(e1, hi2(kv[j]));
                            // the pad column of the accumulator stays zero
                            st4_hint(ap + row * HP,
                                     make_float4(av[j].x + G0.x, av[j].y + G0.y, has1 ? av[j].z + G1.x : 0.f,
                                                 has1 ? av[j].w + G1.y : 0.f),
                                     last ? pol_first : pol_last);
#pragma unroll
                            for (int k = 0; k < MS; ++k) {
                                if (k < M) {
                                    const float2 gy = gsy[(k * f + phy) * L + row], gyd = gsyd[(k * f + phy) * L + row];
                                    U0[k] = cadd(U0[k], cmulc(G0, gy));
                                    U1[k] = cadd(U1[k], cmulc(G1, gy));
                                    V0[k] = cadd(V0[k], cmulc(G0, gyd));
                                    V1[k] = cadd(V1[k], cmulc(G1, gyd));
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < MS; ++k) {
                        if (k < M) {
                            const float2 *gxk = gsx + (k * f + phx) * H, *gxdk = gsxd + (k * f + phx) * H;
                            const float2 gx0 = gxk[c0], gxd0 = gxdk[c0];
                            const float2 gx1 = has1 ? gxk[c1] : make_float2(0.f, 0.f);
                            const float2 gxd1 = has1 ? gxdk[c1] : make_float2(0.f, 0.f);
                            pa[k] += wgt0 * (U0[k].x * gx0.x + U0[k].y * gx0.y) + wgt1 * (U1[k].x * gx1.x + U1[k].y * gx1.y);
                            px[k] += wgt0 * (U0[k].x * gxd0.x + U0[k].y * gxd0.y) +
                                     wgt1 * (U1[k].x * gxd1.x + U1[k].y * gxd1.y);
                            py[k] += wgt0 * (V0[k].x * gx0.x + V0[k].y * gx0.y) + wgt1 * (V1[k].x * gx1.x + V1[k].y * gx1.y);
                        }
                    }
                }
            }
        };
        if (G == 1 && ty2 < RP2) {
            if (M <= 1) adj_one_epoch(std::integral_constant<int, 1>{});
            else adj_one_epoch(std::integral_constant<int, kFftMaxSources>{});
        }
        if (G > 1 && ty < RP) {
            for (int row0 = ty; row0 < L; row0 += rstep) {
                for (int ph = 0; ph < nph; ++ph) {
                    const int phy = ph / f, phx = ph - phy * f;
                    float2 *ap = acc + ph * LHP + tx;
                    float2 kv[kBatch], av[kBatch];
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int g = j & (G - 1), row = row0 + (j >> lgG) * RP;
                        const bool ok = row < L && g < Ge;
                        kv[j] = ok ? ldg_hint(kh + (g * nph + ph) * LHP + row * HP + tx, pol_first) : make_float2(0.f, 0.f);
                        av[j] = (ok && g == 0 && !first) ? ld_hint(ap + row * HP, pol_last) : make_float2(0.f, 0.f);
                    }
                    float2 run = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        const int g = j & (G - 1), row = row0 + (j >> lgG) * RP;
                        if (row < L && g < Ge) {
                            const float2 Gv = cmulc(A[g * EB + row * HP + tx], kv[j]);
                            run = cadd(g == 0 ? av[j] : run, Gv);
                            if (g == Ge - 1) st_hint(ap + row * HP, run, last ? pol_first : pol_last);
                            if (M == 1) {
                                const float2 gx = gsx[g * MfH + phx * H + tx], gy = gsy[g * MfL + phy * L + row];
                                const float2 gxd = gsxd[g * MfH + phx * H + tx], gyd = gsyd[g * MfL + phy * L + row];
                                const float2 s0 = cmul(gx, gy), s1 = cmul(gxd, gy), s2 = cmul(gx, gyd);
                                pa[j] += wgt * (Gv.x * s0.x + Gv.y * s0.y);
                                px[j] += wgt * (Gv.x * s1.x + Gv.y * s1.y);
                                py[j] += wgt * (Gv.x * s2.x + Gv.y * s2.y);
                            }
                        }
                    }
                }
            }
        }
        // fold per epoch (G > 1: batch element j belongs to epoch j mod G) and reduce over the
        // warp in FP32, then across warps as compensated sums below
        if (M > 0) {
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                // q indexes the epoch (G > 1) or the source (G = 1)
                float a = 0.f, bx = 0.f, by = 0.f;
                if (G > 1) {
#pragma unroll
                    for (int j = 0; j < kBatch; ++j) {
                        if ((j & (G - 1)) == q) {
                            a += pa[j];
                            bx += px[j];
                            by += py[j];
                        }
                    }
                } else {
                    a = pa[q];
                    bx = px[q];
                    by = py[q];
                }
                const bool live = G > 1 ? q < Ge : q < M;
                if (live) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        a += __shfl_down_sync(0xffffffffu, a, o);
                        bx += __shfl_down_sync(0xffffffffu, bx, o);
                        by += __shfl_down_sync(0xffffffffu, by, o);
                    }
                    if (lane == 0) {
                        const int g = G > 1 ? q : 0, k = G > 1 ? 0 : q;
                        sh.red[g * nv + 2 + 3 * k][warp] = make_float2(a, 0.f);
                        sh.red[g * nv + 3 + 3 * k][warp] = make_float2(bx, 0.f);
                        sh.red[g * nv + 4 + 3 * k][warp] = make_float2(by, 0.f);
                    }
                }
            }
        }
        __syncthreads();
        // warp v (< Ge nv) sums value v's per-warp partials in a fixed shuffle tree
        if (warp < Ge * nv) {
            const int g = warp / nv, q = warp - g * nv;
            const int cnt = q < 2 ? nsub : nw;
            const float2 part = lane < cnt ? sh.red[warp][lane] : make_float2(0.f, 0.f);
            const FSum tot = fsum_warp(FSum{part.x, part.y});
            if (lane == 0) {
                const double sum = fsum_value(tot);
                const int i = i0 + g;
                if (q == 0) {
                    chi_part[fd.tile_slot + i] = sum;
                } else if (q == 1) {
                    se_part[fd.tile_slot + i] = sum;
                } else {
                    constexpr double kInvL2 = 1.0 / ((double)L * (double)L);
                    const int k = (q - 2) / 3, which = (q - 2) - 3 * k;
                    const long long ps = fd.ps_slot + (long long)i * M + k;
                    const float sc = (float)(sum * kInvL2);
                    if (which == 0) ps_da[ps] = sc;
                    else ps_du[2 * ps + which - 1] = apar[g * M + k] * sc;
                }
            }
        }
        __syncthreads();
    }
}

// Spectra of the folded PSF kernels (computed at set_psfs): item = epoch * f^2 + phase.  The
// phase kernel kappa_phi (Tk x Tk, taps tau_lo .. tau_lo + Tk - 1 on each axis) belongs on the
// L x L circle with tap tau at tau mod L.  It is placed instead at tau - tau_lo (rows and columns
// 0 .. Tk - 1), so that the row passes of fx_fwd2d touch only its ceil(Tk/2) row pairs and Tk
// columns, and the shift is restored on the spectrum (shift theorem):
//   Khat[ky][kx] = W_L^((ky + kx) tau_lo) Khat'[ky][kx],   W_L = exp(-2 pi i / L).
// Written as L rows of pitch HP with the pad column zero.
template <int L>
__device__ __noinline__ void kappa_item_fixed(const FieldDev &fd, const float *__restrict__ kappa,
                                              float2 *__restrict__ khat, int item) {
    using P = Fx<L>;
    constexpr int R2 = P::R2, H = P::H, HP = P::HP, PX = P::PX, EB = P::EBF;
    const int tid = threadIdx.x, nt = blockDim.x;
    float2 *A = fx_dyn, *B = fx_dyn + EB, *TWL = B + EB, *tw = TWL + L;
    for (int n = tid; n < L; n += nt) {
        tw[n] = fd.fft_tw[n];
        TWL[n] = fd.fft_tw[(n % R2) * (n / R2)];
    }
    const int nph = fd.f * fd.f, i = item / nph, ph = item - i * nph;
    const int Tk = fd.Tk, np = (Tk + 1) / 2;
    const float *kap = kappa + ((long long)i * nph + ph) * Tk * Tk;
    for (int t = tid; t < np * Tk; t += nt) {
        const int pr = t / Tk, x = t - pr * Tk;
        const float v0 = kap[(2 * pr) * Tk + x];
        const float v1 = 2 * pr + 1 < Tk ? kap[(2 * pr + 1) * Tk + x] : 0.f;
        A[pr * PX + x] = make_float2(v0, v1);
    }
    __syncthreads();
    fx_fwd2d<L>(A, B, EB, 1, np, 1.f / (float)np, Tk, TWL);
    const int sh = ((fd.tau_lo % L) + L) % L;  // tau_lo mod L
    float2 *out = khat + ((long long)i * nph + ph) * L * HP;
    for (int idx = tid; idx < L * HP; idx += nt) {
        const int ky = idx / HP, kx = idx - ky * HP;
        out[idx] = kx < H ? cmul(A[idx], tw[((ky + kx) * sh) % L]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

#define SR_FX_SIZES(X) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(60) X(64) X(72) X(80) X(96) X(100) X(108) X(120) X(128) X(144)

__global__ void __launch_bounds__(kFftThreads, 1)
fft_kappa_fixed_kernel(FieldDev fd, const float *__restrict__ kappa, float2 *__restrict__ khat) {
    const int n_items = fd.E * fd.f * fd.f;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        switch (fd.fft_L) {
#define SR_FX_KCASE(LL)                                  \
    case LL:                                             \
        kappa_item_fixed<LL>(fd, kappa, khat, item);     \
        break;
            SR_FX_SIZES(SR_FX_KCASE)
#undef SR_FX_KCASE
            default:
                break;  // not reached: transform sizes come from the list
        }
    }
}

// The kernel spectra of many problems in one launch: items[j] = (table entry, epoch * f^2 + phase);
// every block takes items in turn (the spectra live at each entry's fft_khat).
__global__ void __launch_bounds__(kFftThreads, 1)
fft_kappa_fixed_batch_kernel(const FieldDev *__restrict__ fields, const int2 *__restrict__ items, int n_items) {
    for (int j = blockIdx.x; j < n_items; j += gridDim.x) {
        const int2 it = items[j];
        const FieldDev &fd = fields[it.x];
        float2 *khat = const_cast<float2 *>(fd.fft_khat);
        switch (fd.fft_L) {
#define SR_FX_BCASE(LL)                                      \
    case LL:                                                 \
        kappa_item_fixed<LL>(fd, fd.kappa, khat, it.y);      \
        break;
            SR_FX_SIZES(SR_FX_BCASE)
#undef SR_FX_BCASE
            default:
                break;
        }
    }
}

__global__ void __launch_bounds__(kFftThreads, 1)
fft_chunk_fixed_kernel(const FieldDev *__restrict__ fields, const int4 *__restrict__ items, int n_items,
                       int *__restrict__ counter, const float *__restrict__ params,
                       const float2 *__restrict__ hhat_all, float2 *__restrict__ acc_all,
                       double *__restrict__ chi_part, double *__restrict__ se_part, float *__restrict__ ps_da,
                       float *__restrict__ ps_du) {
    for (;;) {
        if (threadIdx.x == 0) fx_sh.item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = fx_sh.item;
        if (it >= n_items) break;
        const int4 item = items[it];
        const FieldDev &fd = fields[item.x];
        switch (fd.fft_L) {
#define SR_FX_CASE(LL)                                                                                          \
    case LL:                                                                                                    \
        chunk_item_fixed<LL>(fd, item, params, hhat_all, acc_all, chi_part, se_part, ps_da, ps_du);          \
        break;
            SR_FX_SIZES(SR_FX_CASE)
#undef SR_FX_CASE
            default:
                break;  // not reached: the host only builds items for sizes in the list
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
bool fft_fixed_size(int L) {
    switch (L) {
#define SR_FX_OK(LL) case LL:
        SR_FX_SIZES(SR_FX_OK)
#undef SR_FX_OK
        return true;
        default:
            return false;
    }
}

int fft_fixed_next(int need) {
    static const int sizes[] = {
#define SR_FX_LIST(LL) LL,
        SR_FX_SIZES(SR_FX_LIST)
#undef SR_FX_LIST
    };
    for (int L : sizes)
        if (L >= need) return L;
    return 0;
}

// Elements (float2) of each of the two per-epoch buffers: the largest of the three layouts.
int fft_fixed_epoch_buffer(int L, int N) {
    const int R1 = fx_r1(L), R2 = L / R1;
    const int S = (R2 & 1) ? R2 : R2 + 1;
    const int np = (N + 1) / 2;
    int eb = std::max(np * L, np * R1 * S);
    eb = std::max(eb, L * (L / 2 + 2));  // the spectrum, rows padded to an even pitch
    return (eb + 1) & ~1;  // keeps every buffer 16-byte aligned
}

int fft_fixed_smem_bytes(int L, int N, int M, int f, int G) {
    const int H = L / 2 + 1;
    return (2 * G * fft_fixed_epoch_buffer(L, N) + 2 * L + 2 * G * M * f * (H + L)) * (int)sizeof(float2);
}

sr_status configure_fft_fixed(int optin, int *limit) {
    float2 tw[kDtwTotal];
    for (int R : {6, 8, 9, 10, 12, 16})
        for (int m = 0; m < R; ++m) {
            const double a = -2.0 * M_PI * (double)m / (double)R;
            tw[dtw_off(R) + m] = make_float2((float)cos(a), (float)sin(a));
        }
    SR_CUDA(cudaMemcpyToSymbol(c_dtw, tw, sizeof(tw)));
    cudaFuncAttributes a;
    SR_CUDA(cudaFuncGetAttributes(&a, fft_chunk_fixed_kernel));
    const int dyn = optin - (int)a.sharedSizeBytes;
    SR_CUDA(cudaFuncSetAttribute(fft_chunk_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    *limit = dyn;
    SR_CUDA(cudaFuncGetAttributes(&a, fft_kappa_fixed_kernel));
    SR_CUDA(cudaFuncSetAttribute(fft_kappa_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)a.sharedSizeBytes));
    SR_CUDA(cudaFuncGetAttributes(&a, fft_kappa_fixed_batch_kernel));
    SR_CUDA(cudaFuncSetAttribute(fft_kappa_fixed_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)a.sharedSizeBytes));
    return SR_OK;
}

static int kappa_fixed_smem(int L) {
    switch (L) {
#define SR_FX_KSMEM(LL) \
    case LL:            \
        return (2 * Fx<LL>::EBF + 2 * LL) * (int)sizeof(float2);
        SR_FX_SIZES(SR_FX_KSMEM)
#undef SR_FX_KSMEM
        default:
            return 0;
    }
}

// Threads of a kernel-spectra block: one per work item of the widest pass (the column passes,
// H * max(R1, R2)), in whole warps, at most kFftThreads: small transforms then pack several
// blocks per SM instead of leaving most of a full-size block idle.
static int kappa_fixed_threads(int L) {
    switch (L) {
#define SR_FX_KTHR(LL)                                                                       \
    case LL: {                                                                               \
        const int w = Fx<LL>::H * (Fx<LL>::R1 > Fx<LL>::R2 ? Fx<LL>::R1 : Fx<LL>::R2);      \
        return std::min(kFftThreads, (w + 31) / 32 * 32);                                    \
    }
        SR_FX_SIZES(SR_FX_KTHR)
#undef SR_FX_KTHR
        default:
            return kFftThreads;
    }
}

sr_status launch_fft_kappa_fixed_batch(const FieldDev *fields, const int2 *items, int n_items, int L, int n_sms,
                                       cudaStream_t st) {
    if (n_items <= 0) return SR_OK;
    const int threads = kappa_fixed_threads(L), smem = kappa_fixed_smem(L);
    int occ = 0;
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fft_kappa_fixed_batch_kernel, threads, smem));
    const int grid = std::min(n_items, std::max(occ, 1) * n_sms);
    fft_kappa_fixed_batch_kernel<<<grid, threads, smem, st>>>(fields, items, n_items);
    return SR_OK;
}

void launch_fft_kappa_fixed(const FieldDev &fd, const float *kappa, float2 *khat, cudaStream_t st) {
    const int n_items = fd.E * fd.f * fd.f;
    fft_kappa_fixed_kernel<<<n_items, kappa_fixed_threads(fd.fft_L), kappa_fixed_smem(fd.fft_L), st>>>(fd, kappa,
                                                                                                     khat);
}

sr_status occupancy_fft_fixed(int smem, int *blocks) {
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fft_chunk_fixed_kernel, kFftThreads, smem));
    return SR_OK;
}

void launch_fft_chunks_fixed(const FieldDev *fields, const int4 *items, int n_items, int *counter,
                             const float *params, const float2 *hhat, float2 *acc, double *chi_part,
                             double *se_part, float *ps_da, float *ps_du, int grid, int smem, cudaStream_t st) {
    fft_chunk_fixed_kernel<<<grid, kFftThreads, smem, st>>>(fields, items, n_items, counter, params, hhat, acc,
                                                            chi_part, se_part, ps_da, ps_du);
}

}  // namespace sr
