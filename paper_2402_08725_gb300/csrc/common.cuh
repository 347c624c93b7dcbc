// Internal definitions shared by the kernels and the host side of the library.
// Not part of the public ABI (see include/starred.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "starred.h"

namespace sr {

// Narrow Gaussian r of Eq. 1 (FWHM 2 fine px): sigma^2 = 1/(2 ln 2), so
// g(v) = exp(-|v|^2/(2 sigma^2)) / (2 pi sigma^2) = (ln 2 / pi) * 2^(-|v|^2).
constexpr float kGaussNorm = 0.220635600152f;      // ln 2 / pi
constexpr float kGaussInvSig2 = 1.386294361120f;   // 1/sigma^2 = 2 ln 2
constexpr float kGauss1Norm = 0.469718639349f;     // 1-D factor: sqrt(ln 2 / pi)
// Point sources are rasterised on a 16 x 16 fine-pixel window starting at
// floor(centre) - 7: every omitted pixel is >= 8 px away, where g < 1e-19 g(0).
constexpr int kWin = 16;
constexpr int kWinLo = 7;
// 1-D Gaussian taps of the PSF-fit blur: |t| <= 8 (g1(8)/g1(0) = 2^-64).
constexpr int kBlurHalf = 8;

constexpr int kMaxScales = 8;
constexpr int kFftThreads = 512;
constexpr int kFftMaxSources = 4;  // point sources per field in the frequency-domain form
constexpr int kFftChunk = 16;      // epochs per work item of the frequency-domain form
constexpr int kThreads = 256;

struct FieldDev {
    int kind;          // SR_DECONV / SR_PSF
    int E, N, f, K, M, J, F;
    int Tk, tau_lo;    // extent and first index of the polyphase folded kernels
    int n_tiles;       // output tiles per epoch (fwd/adj work items)
    float lambda;
    const float *Wd;       // [J-1] prior weights (device, owned by the problem)
    long long param_off;   // offset of the field in the parameter vector
    long long ebuf_off;    // floats, E*N*N residual-weight buffer
    long long gbuf_off;    // floats, E*f*f*N*N per-epoch adjoint images (polyphase layout)
    long long tile_slot;   // first (epoch, tile) slot of the field's partial sums
    long long ps_slot;     // first (epoch, source) slot
    long long l1_slot;     // first (level, chunk) slot of the prior partial sums
    int n_chunks;          // 256-pixel chunks of the F x F grid
    const float *d;        // [E][N][N]
    const float *w;        // [E][N][N] inverse variance (0 = masked)
    const float *kappa;    // [E][f*f][Tk][Tk] folded kernels (DECONV)
    float *starlet;        // [(J + 2)][F][F] scratch planes
    float *psf_s;          // PSF kind: [F][F] narrow PSF s = m + b
    float *psf_tmp;        // PSF kind: [S][3][F][F] row-pass planes (value, d/dx) and adjoint plane
    float *psf_gs;         // PSF kind: [S][F][F] per-star gradient wrt s
    // frequency-domain form (fft_pair.cu); mode 0 = direct tiles, 1 = transforms
    int mode;
    int fft_L;
    const float2 *fft_tw;     // [L] exp(-2 pi i n / L)
    // spectra in global memory are rows of L/2+2 (the last column a zero pad, so that column
    // pairs are 16-byte aligned)
    const float2 *fft_khat;   // [E][f*f][L][L/2+2] transforms of the folded kernels
    long long fft_hhat_off;   // offset of the field's [f*f][L][L/2+2] h spectra in the plan buffer
    long long fft_acc_off;    // float2 offset of the field's chunk accumulators ([f*f][L][L/2+2] each)
    int fft_n_chunks;         // epoch chunks of the field
    int fft_G;                // epoch pairs transformed side by side by the chunk kernel (1, 2 or 4)
    int fft_EB;               // float2 elements of one pair array of the transform kernels
    // point-source prior (Eq. 11, third term): 1 + index of the partner entry (a field's shadow
    // entry in the plan's point-source table, or a shadow entry's field), 0 for none
    int pts;
    // the extended channel moved with each epoch's shift (f_i = T_{f delta_i} h + P_i, bilinear,
    // zero outside; direct form only) and the offset of its shift gradients (2 per epoch)
    int translate;
    long long hs_off;
    // rotated frames: per epoch (cos theta_i, sin theta_i) of the frame's turn about the grid
    // centre (device, owned by the problem), or NULL; direct form only
    const float2 *rot;
    // per-coefficient prior weights [J-1][F][F] (device, owned by the problem), or NULL: the prior
    // is then lambda Wd[j] |w_j| per scale; with a map, lambda Wd[j] Wmap[j][u] |w_j(u)| (Wd = 1,
    // or lambda_pts for a point-source shadow entry)
    const float *Wmap;
};

// Plane j of the weight map (NULL without a map), read once per kernel into a register: the
// field table lives in global memory, where the kernels' stores could alias it.
__device__ __forceinline__ const float *wmap_plane(const FieldDev &fd, int j) {
    return (fd.Wmap && j >= 0) ? fd.Wmap + (long long)j * fd.F * fd.F : nullptr;
}
// The weight of coefficient u of that plane: the map's value, 1 without a map.
__device__ __forceinline__ float wmap_w(const float *__restrict__ wm, long long u) { return wm ? __ldg(wm + u) : 1.f; }

// Whole and fractional parts of the bilinear read of a channel moved by s fine pixels: output u
// reads u + n (weight 1 - t) and u + n + 1 (weight t), n = floor(-s), t = -s - n in [0, 1).
// The reference-frame point seen by fine pixel (ux, uy) of a rotated frame:
// q = u0 + R^T (u - u0 - s), R = [[c, -s], [s, c]] with (c, s) = cs; sh the frame's shift.  One
// code path with explicit fused operations, so that every kernel takes the same cell decisions.
__device__ __forceinline__ float2 frame_point(int F, float2 cs, float2 sh, int ux, int uy) {
    const float u0 = 0.5f * (float)(F - 1);
    const float dx = (float)ux - __fadd_rn(u0, sh.x), dy = (float)uy - __fadd_rn(u0, sh.y);
    return make_float2(__fmaf_rn(cs.y, dy, __fmaf_rn(cs.x, dx, u0)), __fmaf_rn(cs.x, dy, __fmaf_rn(-cs.y, dx, u0)));
}

__device__ __forceinline__ void shift_split(float s, int *n, float *t) {
    const float fl = floorf(-s);
    *n = (int)fl;
    *t = -s - fl;
}

// One output tile of one epoch: rows [y0, y0+h), cols [x0, x0+w) of the data
// grid.  pg = number of thread groups working on different phases at once.
struct TileItem {
    int field;
    int epoch;
    int slot;      // (epoch, tile) partial-sum slot
    short y0, x0, h, w;
    int pg;
};

struct ChunkItem {
    int field;
    int start;     // first pixel (row-major F*F index) of the chunk
    int chunk;     // chunk index within the field
};

// Offset u - centre of fine pixel u from a point source whose fine centre is
// (F-1)/2 + f (c + delta).  The centre can be hundreds of pixels from the origin while the
// offset is a few pixels, so the offset is formed from small quantities: u - (F-1)/2 is exact,
// and each product f*c, f*delta is rounded only together with the small running difference.
__device__ __forceinline__ float src_offset(int u, int F, int f, float c, float delta) {
    const float t = (float)u - 0.5f * (float)(F - 1);
    return fmaf(-(float)f, delta, fmaf(-(float)f, c, t));
}

}  // namespace sr

// --- host-side helpers shared by the .cu files ---------------------------------
namespace sr {
void set_error(const char *fmt, ...);
sr_status cuda_fail(cudaError_t e, const char *what);
}  // namespace sr

#define SR_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::sr::cuda_fail(_e, #call);       \
    } while (0)
