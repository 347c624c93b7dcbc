// Starlet prior lambda ||W o Phi^T h||_1 (Eq. 6, Eq. 11) and its gradient (sm_103a).
//
// Phi^T is the isotropic undecimated B3-spline starlet: c_0 = h, c_{j+1} = H_j c_j with H_j
// the separable filter (1,4,6,4,1)/16 dilated by 2^j (whole-sample mirror borders), and detail
// planes w_{j+1} = c_j - c_{j+1}, j = 0..J-2.  The prior is lambda sum_j W_j sum_u |w_{j+1}[u]|.
// Its gradient is T_0, where T_{J-1} = 0 and
//     T_j = gamma_{j+1} + H_j^T (T_{j+1} - gamma_{j+1}),   gamma_{j+1} = lambda W_j sign(w_{j+1}),
// and H_j^T = (row pass)^T (column pass)^T is evaluated in gather form: each output sums the
// (up to three) input positions that the mirror map sends onto it.
//
// Scratch per field (planes of F*F floats): c_1..c_{J-1} (planes 0..J-2), a spare plane (J-1),
// and two T planes (J, J+1) used alternately; T_0 ends in plane J.
//
// Three ways to run a level, chosen per field (starlet_form):
//  * comb bands (most fields): the rows rho, rho + s, rho + 2 s, ... of level j (step s = 2^j)
//    are one column tap apart, so a block taking 16 consecutive rows of one such comb stages
//    only 20 input rows at any level; otherwise the same as the bands below, whose arithmetic
//    and order it keeps (the column gather's mirror preimages are read from the plane).
//  * bands: one launch per level; a block takes 16 output rows of one field, filters the rows it
//    needs (with their 2 * 2^j-row halo) along x into shared memory, then along y.  The adjoint
//    propagates V_j = T_j - gamma_j instead of T_j (V_{J-1} = -gamma_{J-1} is formed while
//    loading), so that its column pass reads one plane per tap; the signs are taken from the c
//    planes once per output pixel.
//  * tiles (fields too wide for comb bands of whole rows): the comb bands on 128 columns, with
//    the 2 * 2^j halo along x (the forward reads its row taps from the c plane directly; the
//    adjoint stages the V rows and the column-adjoint values of the tile's columns and halo,
//    which hold every mirror preimage its row gather reaches).
// Fields deeper than a level skip it.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ffsum.cuh"
#include "kernels.cuh"

namespace sr {

__constant__ float kB3[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};

constexpr int kBandRows = 16;                  // output rows per block in the band kernels
constexpr int kBandSmemBytes = 100 * 1024;     // shared memory of a band block (two per SM)

// Whether a field runs its levels as bands: the deepest level's adjoint (2 * 16 + 4 * 2^(J-2)
// rows of F floats) fits the budget.
__host__ __device__ inline bool starlet_banded(int F, int J) {
    const long long s = 1LL << (J - 2);
    return (2LL * kBandRows + 4 * s) * F * (long long)sizeof(float) <= kBandSmemBytes;
}

constexpr int kTileCols = 128;                 // output columns per block in the tile kernels
constexpr int kTileSmemBytes = 160 * 1024;     // shared memory of a tile block at its deepest level

// Comb bands: at level j (step s = 2^j) the rows congruent to rho modulo s form a comb whose rows
// are s apart, which is exactly the spacing of the level's column taps; a block takes 16
// consecutive rows of one comb and stages 20 (two more on each side) instead of 16 + 4 s.
constexpr int kCombRows = 16;  // rows of a comb per block (fewer for small tables, see comb_rows)
constexpr int kCombMaxF = kBandSmemBytes / ((2 * kCombRows + 4) * (int)sizeof(float));  // adjoint budget
// Blocks of level j: s combs of ceil(ceil(F / s) / cr) chunks each.
__host__ __device__ inline int comb_chunks(int F, int s, int cr = kCombRows) {
    return ((F + s - 1) / s + cr - 1) / cr;
}
// The prior's partial sums of a comb-band level are kept per group of 4 consecutive comb rows
// (whatever the rows per block), so that the sum does not depend on the block shape.
constexpr int kCombGroup = 4;
// A field runs its levels as comb bands when a row of the adjoint's staging fits the budget and
// every level's row groups fit the prior partial-sum slots of a level (one per 256 pixels).
__host__ __device__ inline bool starlet_combed(int F, int J) {
    if (F > kCombMaxF) return false;
    const int slots = (F * F + 255) / 256;
    for (int j = 0; j <= J - 2; ++j)
        if ((1 << j) * comb_chunks(F, 1 << j, kCombGroup) > slots) return false;
    return true;
}
// Tiles (grids too wide for the comb bands): comb rows as above by 128 columns with the 2 s halo
// along x.  Shared memory (floats) at level j: the forward's row-filtered rows (20 rows of 128),
// the adjoint's V rows and column-adjoint rows (20 and 16 rows of 128 + 4 s).
__host__ __device__ inline long long tile_fwd_floats(int) { return (long long)(kCombRows + 4) * kTileCols; }
__host__ __device__ inline long long tile_adj_floats(int j) {
    const long long s = 1LL << j;
    return (2LL * kCombRows + 4) * (kTileCols + 4 * s);
}
// Whether a field too wide for the comb bands runs as tiles: its deepest level fits the budget
// and every level's (4-row group, column tile) partial sums fit the slots of a level.
__host__ __device__ inline bool starlet_tiled(int F, int J) {
    if (starlet_banded(F, J) || tile_adj_floats(J - 2) * (long long)sizeof(float) > kTileSmemBytes) return false;
    const int slots = (F * F + 255) / 256, nbx = (F + kTileCols - 1) / kTileCols;
    for (int j = 0; j <= J - 2; ++j)
        if ((long long)(1 << j) * comb_chunks(F, 1 << j, kCombGroup) * nbx > slots) return false;
    return true;
}

// 0 bands, 1 tiles, 3 comb bands; 2: none (no shape of at most 8 scales on a grid of at most
// 32768 pixels comes here; sr_create_problem rejects one that would)
__host__ __device__ inline int starlet_form(int F, int J) {
    return starlet_combed(F, J) ? 3 : starlet_banded(F, J) ? 0 : starlet_tiled(F, J) ? 1 : 2;
}

__device__ __forceinline__ int mirror_at(int t, int F) { return t < 0 ? -t : (t > F - 1 ? 2 * (F - 1) - t : t); }

__device__ __forceinline__ const float *c_plane(const FieldDev &fd, const float *params, int j) {
    return j == 0 ? params + fd.param_off : fd.starlet + (long long)(j - 1) * fd.F * fd.F;
}
__device__ __forceinline__ float *t_plane(const FieldDev &fd, int j) {
    return fd.starlet + (long long)(fd.J + (j & 1)) * fd.F * fd.F;
}

// (H^T y)[n] along one axis: sum over taps m and over the mirror preimages of n.  Away from the
// edges (2 step < n < F - 1 - 2 step) every tap is direct and no preimage exists: the same sum
// without the tests.
__device__ __forceinline__ float adj_1d(const float *__restrict__ y, int n, int F, int step, int stride) {
    float acc = 0.f;
    if (n > 2 * step && n < F - 1 - 2 * step) {
#pragma unroll
        for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * y[(long long)(n - m * step) * stride];
        return acc;
    }
#pragma unroll
    for (int m = -2; m <= 2; ++m) {
        const float b = kB3[m + 2];
        const int k1 = n - m * step;
        if (k1 >= 0 && k1 < F) acc += b * y[(long long)k1 * stride];
        if (n > 0) {
            const int k2 = -n - m * step;
            if (k2 >= 0 && k2 < F) acc += b * y[(long long)k2 * stride];
        }
        if (n < F - 1) {
            const int k3 = 2 * (F - 1) - n - m * step;
            if (k3 >= 0 && k3 < F) acc += b * y[(long long)k3 * stride];
        }
    }
    return acc;
}

// Forward level j as bands: c_{j+1} = Col_j Row_j c_j on rows [y0, y0 + 16) and the prior
// partial lambda W_j sum |c_j - c_{j+1}| of the band.  Block (b, field).
template <bool MAP>
__global__ void __launch_bounds__(256)
starlet_band_fwd_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                        double *__restrict__ l1_part, int j) {
    extern __shared__ float sb[];
    __shared__ float2 s_red[8];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 0) return;
    const int b = blockIdx.x, y0 = b * kBandRows;
    if (y0 >= F) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int s = 1 << j, Tr = min(kBandRows, F - y0), r0 = y0 - 2 * s;
    // rows r0 .. y0 + Tr - 1 + 2s (mirrored: one reflection, as 2 s <= F - 1), filtered along x
    const int R = Tr + 4 * s;
    const float *cj = c_plane(fd, params, j);
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr;
    for (int i = warp; i < R; i += nwarp) {
        const float *row = cj + (long long)mirror_at(r0 + i, F) * F;
        float *dst = sb + (long long)i * F;
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
            if (x >= 2 * s && x <= F - 1 - 2 * s) {  // all taps inside: no mirror
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[x + n * s];
            } else {
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[mirror_at(x + n * s, F)];
            }
            dst[x] = acc;
        }
    }
    __syncthreads();
    float *cn = fd.starlet + (long long)j * F * F;  // c_{j+1}
    // |w| summed in FP32 along a row, the rows as compensated sums
    FSum l1 = fsum_zero();
    for (int yy = warp; yy < Tr; yy += nwarp) {
        const long long ro = (long long)(y0 + yy) * F;
        float l1_row = 0.f;
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
#pragma unroll
            for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * sb[(long long)(yy + 2 * s + m * s) * F + x];
            cn[ro + x] = acc;
            l1_row += fabsf(cj[ro + x] - acc) * wmap_w(wm1, ro + x);
        }
        l1 = fsum_add(l1, l1_row);
    }
    l1 = fsum_warp(l1);
    if (lane == 0) s_red[warp] = make_float2(l1.hi, l1.lo);
    __syncthreads();
    const long long base = fd.l1_slot + (long long)j * fd.n_chunks;
    if (threadIdx.x == 0) {
        FSum t = fsum_zero();
        for (int w = 0; w < nwarp; ++w) t = fsum_add(t, FSum{s_red[w].x, s_red[w].y});
        l1_part[base + b] = (double)fd.lambda * (double)fd.Wd[j] * fsum_value(t);
    }
    if (b == 0) {  // the level's remaining partial-sum slots (one per 256-pixel chunk) stay zero
        const int nb = (F + kBandRows - 1) / kBandRows;
        for (int c = nb + threadIdx.x; c < fd.n_chunks; c += blockDim.x) l1_part[base + c] = 0.0;
    }
}

__device__ __forceinline__ float gamma_of(float wv, float lw) { return wv > 0.f ? lw : (wv < 0.f ? -lw : 0.f); }

// Adjoint level j as bands: T_j = gamma_{j+1} + Row_j^T Col_j^T V_{j+1} on rows [y0, y0 + 16),
// written as V_j = T_j - gamma_j (j >= 1) or T_0 (j = 0) into plane J + (j & 1).
template <bool MAP>
__global__ void __launch_bounds__(256, 4)  // at most 64 registers: four blocks per SM
starlet_band_adj_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int j) {
    extern __shared__ float sb[];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 0) return;
    const int b = blockIdx.x, y0 = b * kBandRows;
    if (y0 >= F) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int s = 1 << j, Tr = min(kBandRows, F - y0);
    // every row the column gather below can reach (mirror preimages included)
    const int vlo = max(0, y0 - 2 * s), vhi = min(F, y0 + Tr + 2 * s);
    float *vb = sb, *tb = sb + (long long)(kBandRows + 4 * s) * F;
    const float lw1 = fd.lambda * fd.Wd[j];
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr, *wm0 = MAP ? wmap_plane(fd, j - 1) : nullptr;
    const float *cj = c_plane(fd, params, j), *cn = fd.starlet + (long long)j * F * F;  // c_j, c_{j+1}
    const bool top = j + 1 == J - 1;
    const float *Vn = fd.starlet + (long long)(J + ((j + 1) & 1)) * F * F;
    for (int i = warp; i < vhi - vlo; i += nwarp) {
        const long long ro = (long long)(vlo + i) * F;
        for (int x = lane; x < F; x += 32)
            vb[(long long)i * F + x] =
                top ? 0.f - gamma_of(cj[ro + x] - cn[ro + x], lw1 * wmap_w(wm1, ro + x)) : Vn[ro + x];
    }
    __syncthreads();
    for (int yy = warp; yy < Tr; yy += nwarp) {
        const int y = y0 + yy;
        const bool inner = y > 2 * s && y < F - 1 - 2 * s;  // direct taps only (no mirror preimage)
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
            if (inner) {
#pragma unroll
                for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * vb[(long long)(y - m * s - vlo) * F + x];
                tb[(long long)yy * F + x] = acc;
                continue;
            }
#pragma unroll
            for (int m = -2; m <= 2; ++m) {
                const float bm = kB3[m + 2];
                const int k1 = y - m * s;
                if (k1 >= 0 && k1 < F) acc += bm * vb[(long long)(k1 - vlo) * F + x];
                const int k2 = -y - m * s;
                if (y > 0 && k2 >= 0 && k2 < F) acc += bm * vb[(long long)(k2 - vlo) * F + x];
                const int k3 = 2 * (F - 1) - y - m * s;
                if (y < F - 1 && k3 >= 0 && k3 < F) acc += bm * vb[(long long)(k3 - vlo) * F + x];
            }
            tb[(long long)yy * F + x] = acc;
        }
    }
    __syncthreads();
    const float lw0 = j >= 1 ? fd.lambda * fd.Wd[j - 1] : 0.f;
    const float *cjm = j >= 1 ? c_plane(fd, params, j - 1) : cj;  // c_{j-1}
    float *out = fd.starlet + (long long)(J + (j & 1)) * F * F;
    for (int yy = warp; yy < Tr; yy += nwarp) {
        const long long ro = (long long)(y0 + yy) * F;
        const float *trow = tb + (long long)yy * F;
        for (int x = lane; x < F; x += 32) {
            const float acc = adj_1d(trow, x, F, s, 1);
            const float tj = gamma_of(cj[ro + x] - cn[ro + x], lw1 * wmap_w(wm1, ro + x)) + acc;
            out[ro + x] = j >= 1 ? tj - gamma_of(cjm[ro + x] - cj[ro + x], lw0 * wmap_w(wm0, ro + x)) : tj;
        }
    }
}

// Forward level j as comb bands: block b takes rows y_t = rho + s (k0 + t), t < cr, of comb rho,
// filters rows rho + s (k0 - 2 + i), i < cr + 4 (mirrored), along x into shared memory, then along
// y: each output row's five taps are staged rows t .. t + 4.  The same values, in the same order,
// as the bands.  Block (b, field), b = rho * nk + k0 / cr.
template <bool MAP>
__global__ void __launch_bounds__(256)
starlet_comb_fwd_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                        double *__restrict__ l1_part, int j, int cr) {
    extern __shared__ float sb[];
    __shared__ float2 s_row[kCombRows];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 3) return;
    const int s = 1 << j, nk = comb_chunks(F, s, cr), b = blockIdx.x;
    if (b >= s * nk) return;
    const int rho = b / nk, k0 = (b - rho * nk) * cr;
    const int Tr = max(0, min(cr, (F - rho + s - 1) / s - k0));  // rows of the comb in the grid
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const float *cj = c_plane(fd, params, j);
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr;
    const int R = Tr > 0 ? Tr + 4 : 0;
    for (int i = warp; i < R; i += nwarp) {
        const float *row = cj + (long long)mirror_at(rho + s * (k0 - 2 + i), F) * F;
        float *dst = sb + (long long)i * F;
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
            if (x >= 2 * s && x <= F - 1 - 2 * s) {  // all taps inside: no mirror
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[x + n * s];
            } else {
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[mirror_at(x + n * s, F)];
            }
            dst[x] = acc;
        }
    }
    __syncthreads();
    float *cn = fd.starlet + (long long)j * F * F;  // c_{j+1}
    for (int t = warp; t < Tr; t += nwarp) {
        const long long ro = (long long)(rho + s * (k0 + t)) * F;
        float l1_row = 0.f;
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
#pragma unroll
            for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * sb[(long long)(t + 2 + m) * F + x];
            cn[ro + x] = acc;
            l1_row += fabsf(cj[ro + x] - acc) * wmap_w(wm1, ro + x);
        }
        const FSum r = fsum_warp(FSum{l1_row, 0.f});  // the row's sum (lanes in a fixed tree)
        if (lane == 0) s_row[t] = make_float2(r.hi, r.lo);
    }
    __syncthreads();
    // the partial of each group of 4 comb rows (its rows' sums in order) into the group's slot
    const int nk4 = comb_chunks(F, s, kCombGroup), g0 = k0 / kCombGroup;
    const long long base = fd.l1_slot + (long long)j * fd.n_chunks;
    for (int g = threadIdx.x; g < cr / kCombGroup; g += blockDim.x) {
        if (g0 + g >= nk4) break;
        FSum a = fsum_zero();
        for (int t = kCombGroup * g; t < min(kCombGroup * (g + 1), Tr); ++t)
            a = fsum_add(a, FSum{s_row[t].x, s_row[t].y});
        l1_part[base + (long long)rho * nk4 + g0 + g] = (double)fd.lambda * (double)fd.Wd[j] * fsum_value(a);
    }
    if (b == 0)  // the level's remaining partial-sum slots stay zero
        for (int c = s * nk4 + threadIdx.x; c < fd.n_chunks; c += blockDim.x) l1_part[base + c] = 0.0;
}

// Adjoint level j as comb bands: T_j = gamma_{j+1} + Row_j^T Col_j^T V_{j+1} on the comb rows of
// block b, written as V_j = T_j - gamma_j (j >= 1) or T_0 (j = 0) into plane J + (j & 1).  The
// direct taps y - m s of the column gather are the staged comb rows t - m + 2; its mirror
// preimages (rows within 2 s of the grid's edges, in other combs) are read from the plane.  The
// same values, in the same order, as the bands.
template <bool MAP>
__global__ void __launch_bounds__(256, 4)  // at most 64 registers: four blocks per SM
starlet_comb_adj_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int j, int cr) {
    extern __shared__ float sb[];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 3) return;
    const int s = 1 << j, nk = comb_chunks(F, s, cr), b = blockIdx.x;
    if (b >= s * nk) return;
    const int rho = b / nk, k0 = (b - rho * nk) * cr;
    const int Tr = max(0, min(cr, (F - rho + s - 1) / s - k0));
    if (Tr == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    float *vb = sb, *tb = sb + (long long)(cr + 4) * F;
    const float lw1 = fd.lambda * fd.Wd[j];
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr, *wm0 = MAP ? wmap_plane(fd, j - 1) : nullptr;
    const float *cj = c_plane(fd, params, j), *cn = fd.starlet + (long long)j * F * F;  // c_j, c_{j+1}
    const bool top = j + 1 == J - 1;
    const float *Vn = fd.starlet + (long long)(J + ((j + 1) & 1)) * F * F;
    // V_{j+1} (for the top level -gamma_{J-1}, formed on the fly) at row r, column x
    auto vval = [&](int r, int x) {
        const long long o = (long long)r * F + x;
        return top ? 0.f - gamma_of(cj[o] - cn[o], lw1 * wmap_w(wm1, o)) : Vn[o];
    };
    for (int i = warp; i < Tr + 4; i += nwarp) {
        const int r = rho + s * (k0 - 2 + i);
        if (r < 0 || r >= F) continue;  // never read: the gather tests the same range
        for (int x = lane; x < F; x += 32) vb[(long long)i * F + x] = vval(r, x);
    }
    __syncthreads();
    for (int t = warp; t < Tr; t += nwarp) {
        const int y = rho + s * (k0 + t);
        const bool inner = y > 2 * s && y < F - 1 - 2 * s;  // direct taps only (no mirror preimage)
        for (int x = lane; x < F; x += 32) {
            float acc = 0.f;
            if (inner) {
#pragma unroll
                for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * vb[(long long)(t - m + 2) * F + x];
                tb[(long long)t * F + x] = acc;
                continue;
            }
#pragma unroll
            for (int m = -2; m <= 2; ++m) {
                const float bm = kB3[m + 2];
                const int k1 = y - m * s;
                if (k1 >= 0 && k1 < F) acc += bm * vb[(long long)(t - m + 2) * F + x];
                const int k2 = -y - m * s;
                if (y > 0 && k2 >= 0 && k2 < F) acc += bm * vval(k2, x);
                const int k3 = 2 * (F - 1) - y - m * s;
                if (y < F - 1 && k3 >= 0 && k3 < F) acc += bm * vval(k3, x);
            }
            tb[(long long)t * F + x] = acc;
        }
    }
    __syncthreads();
    const float lw0 = j >= 1 ? fd.lambda * fd.Wd[j - 1] : 0.f;
    const float *cjm = j >= 1 ? c_plane(fd, params, j - 1) : cj;  // c_{j-1}
    float *out = fd.starlet + (long long)(J + (j & 1)) * F * F;
    for (int t = warp; t < Tr; t += nwarp) {
        const long long ro = (long long)(rho + s * (k0 + t)) * F;
        const float *trow = tb + (long long)t * F;
        for (int x = lane; x < F; x += 32) {
            const float acc = adj_1d(trow, x, F, s, 1);
            const float tj = gamma_of(cj[ro + x] - cn[ro + x], lw1 * wmap_w(wm1, ro + x)) + acc;
            out[ro + x] = j >= 1 ? tj - gamma_of(cjm[ro + x] - cj[ro + x], lw0 * wmap_w(wm0, ro + x)) : tj;
        }
    }
}

// Forward level j as tiles: the comb-band forward on the columns [x0, x0 + 128) (the row taps read
// from c_j directly).  Block (t, field), t = (rho * nk + k0 / 16) * nbx + x0 / 128; the prior's
// partial sums per (4-row comb group, column tile).
template <bool MAP>
__global__ void __launch_bounds__(256)
starlet_tile_fwd_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                        double *__restrict__ l1_part, int j) {
    extern __shared__ float sb[];
    __shared__ float2 s_row[kCombRows];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 1) return;
    const int s = 1 << j, nk = comb_chunks(F, s), nbx = (F + kTileCols - 1) / kTileCols;
    const int t0 = blockIdx.x;
    if (t0 >= s * nk * nbx) return;
    const int cb = t0 / nbx, bx = t0 - cb * nbx, x0 = bx * kTileCols, Tc = min(kTileCols, F - x0);
    const int rho = cb / nk, k0 = (cb - rho * nk) * kCombRows;
    const int Tr = max(0, min(kCombRows, (F - rho + s - 1) / s - k0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const float *cj = c_plane(fd, params, j);
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr;
    const int R = Tr > 0 ? Tr + 4 : 0;
    for (int i = warp; i < R; i += nwarp) {
        const float *row = cj + (long long)mirror_at(rho + s * (k0 - 2 + i), F) * F;
        float *dst = sb + (long long)i * kTileCols;
        for (int xx = lane; xx < Tc; xx += 32) {
            const int x = x0 + xx;
            float acc = 0.f;
            if (x >= 2 * s && x <= F - 1 - 2 * s) {  // all taps inside: no mirror
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[x + n * s];
            } else {
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * row[mirror_at(x + n * s, F)];
            }
            dst[xx] = acc;
        }
    }
    __syncthreads();
    float *cn = fd.starlet + (long long)j * F * F;  // c_{j+1}
    for (int t = warp; t < Tr; t += nwarp) {
        const long long ro = (long long)(rho + s * (k0 + t)) * F;
        float l1_row = 0.f;
        for (int xx = lane; xx < Tc; xx += 32) {
            const int x = x0 + xx;
            float acc = 0.f;
#pragma unroll
            for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * sb[(long long)(t + 2 + m) * kTileCols + xx];
            cn[ro + x] = acc;
            l1_row += fabsf(cj[ro + x] - acc) * wmap_w(wm1, ro + x);
        }
        const FSum r = fsum_warp(FSum{l1_row, 0.f});
        if (lane == 0) s_row[t] = make_float2(r.hi, r.lo);
    }
    __syncthreads();
    const int nk4 = comb_chunks(F, s, kCombGroup), g0 = k0 / kCombGroup;
    const long long base = fd.l1_slot + (long long)j * fd.n_chunks;
    for (int g = threadIdx.x; g < kCombRows / kCombGroup; g += blockDim.x) {
        if (g0 + g >= nk4) break;
        FSum a = fsum_zero();
        for (int t = kCombGroup * g; t < min(kCombGroup * (g + 1), Tr); ++t)
            a = fsum_add(a, FSum{s_row[t].x, s_row[t].y});
        l1_part[base + ((long long)rho * nk4 + g0 + g) * nbx + bx] =
            (double)fd.lambda * (double)fd.Wd[j] * fsum_value(a);
    }
    if (t0 == 0)  // the level's remaining partial-sum slots stay zero
        for (long long c = (long long)s * nk4 * nbx + threadIdx.x; c < fd.n_chunks; c += blockDim.x)
            l1_part[base + c] = 0.0;
}

// Adjoint level j as tiles: the comb-band adjoint on the columns [x0, x0 + 128): the V rows and
// the column-adjoint values are staged over the tile's columns and their 2 s halo (clipped to the
// grid), which hold every mirror preimage of the row gather; the column gather's mirror
// preimages are read from the plane.
template <bool MAP>
__global__ void __launch_bounds__(256)
starlet_tile_adj_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params, int j) {
    extern __shared__ float sb[];
    const FieldDev &fd = fields[blockIdx.y];
    const int F = fd.F, J = fd.J;
    if (j > J - 2 || starlet_form(F, J) != 1) return;
    const int s = 1 << j, nk = comb_chunks(F, s), nbx = (F + kTileCols - 1) / kTileCols;
    const int t0 = blockIdx.x;
    if (t0 >= s * nk * nbx) return;
    const int cb = t0 / nbx, bx = t0 - cb * nbx, x0 = bx * kTileCols, Tc = min(kTileCols, F - x0);
    const int rho = cb / nk, k0 = (cb - rho * nk) * kCombRows;
    const int Tr = max(0, min(kCombRows, (F - rho + s - 1) / s - k0));
    if (Tr == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int xlo = max(0, x0 - 2 * s), xhi = min(F, x0 + Tc + 2 * s), W = xhi - xlo;
    const int WP = kTileCols + 4 * s;  // row pitch of both staged arrays
    float *vb = sb, *tb = sb + (long long)(kCombRows + 4) * WP;
    const float lw1 = fd.lambda * fd.Wd[j];
    const float *wm1 = MAP ? wmap_plane(fd, j) : nullptr, *wm0 = MAP ? wmap_plane(fd, j - 1) : nullptr;
    const float *cj = c_plane(fd, params, j), *cn = fd.starlet + (long long)j * F * F;  // c_j, c_{j+1}
    const bool top = j + 1 == J - 1;
    const float *Vn = fd.starlet + (long long)(J + ((j + 1) & 1)) * F * F;
    auto vval = [&](int r, int x) {
        const long long o = (long long)r * F + x;
        return top ? 0.f - gamma_of(cj[o] - cn[o], lw1 * wmap_w(wm1, o)) : Vn[o];
    };
    for (int i = warp; i < Tr + 4; i += nwarp) {
        const int r = rho + s * (k0 - 2 + i);
        if (r < 0 || r >= F) continue;  // never read: the gather tests the same range
        for (int xx = lane; xx < W; xx += 32) vb[(long long)i * WP + xx] = vval(r, xlo + xx);
    }
    __syncthreads();
    for (int t = warp; t < Tr; t += nwarp) {
        const int y = rho + s * (k0 + t);
        const bool inner = y > 2 * s && y < F - 1 - 2 * s;  // direct taps only (no mirror preimage)
        for (int xx = lane; xx < W; xx += 32) {
            float acc = 0.f;
            if (inner) {
#pragma unroll
                for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * vb[(long long)(t - m + 2) * WP + xx];
                tb[(long long)t * WP + xx] = acc;
                continue;
            }
            const int x = xlo + xx;
#pragma unroll
            for (int m = -2; m <= 2; ++m) {
                const float bm = kB3[m + 2];
                const int k1 = y - m * s;
                if (k1 >= 0 && k1 < F) acc += bm * vb[(long long)(t - m + 2) * WP + xx];
                const int k2 = -y - m * s;
                if (y > 0 && k2 >= 0 && k2 < F) acc += bm * vval(k2, x);
                const int k3 = 2 * (F - 1) - y - m * s;
                if (y < F - 1 && k3 >= 0 && k3 < F) acc += bm * vval(k3, x);
            }
            tb[(long long)t * WP + xx] = acc;
        }
    }
    __syncthreads();
    const float lw0 = j >= 1 ? fd.lambda * fd.Wd[j - 1] : 0.f;
    const float *cjm = j >= 1 ? c_plane(fd, params, j - 1) : cj;  // c_{j-1}
    float *out = fd.starlet + (long long)(J + (j & 1)) * F * F;
    for (int t = warp; t < Tr; t += nwarp) {
        const long long ro = (long long)(rho + s * (k0 + t)) * F;
        const float *trow = tb + (long long)t * WP - xlo;  // indexed by the grid column
        for (int xx = lane; xx < Tc; xx += 32) {
            const int x = x0 + xx;
            const float acc = adj_1d(trow, x, F, s, 1);
            const float tj = gamma_of(cj[ro + x] - cn[ro + x], lw1 * wmap_w(wm1, ro + x)) + acc;
            out[ro + x] = j >= 1 ? tj - gamma_of(cjm[ro + x] - cj[ro + x], lw0 * wmap_w(wm0, ro + x)) : tj;
        }
    }
}

int starlet_field_form(int F, int J) { return starlet_form(F, J); }

int starlet_forms_single(int F, int J, bool map) {
    static std::atomic<int> sms_cached{0};  // the SM count, looked up once (any thread may store it)
    int sms = sms_cached.load(std::memory_order_relaxed);
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                       cudaSuccess || sms <= 0)
            sms = 1;
        sms_cached.store(sms, std::memory_order_relaxed);
    }
    const int forms = (1 << starlet_form(F, J)) | (map ? kStarletMapBit : 0);
    return forms | starlet_comb_rows_bits(&F, &J, 1, sms);
}

int starlet_comb_rows_of(int forms) { return (forms & kStarletRows8) ? 8 : (forms & kStarletRows4) ? 4 : kCombRows; }

// Rows per comb block for a table of comb-band fields (F, J of each): 16, or 8 or 4 when the
// table's level-0 blocks would not fill twice the SMs.  The results do not depend on it (the
// prior's partial sums are kept per 4-row group).  Returns the forms bit to add (0 for 16 rows).
int starlet_comb_rows_bits(const int *F, const int *J, int n, int n_sms) {
    long long blocks = 0;
    for (int i = 0; i < n; ++i)
        if (starlet_form(F[i], J[i]) == 3) blocks += comb_chunks(F[i], 1);
    if (blocks == 0 || blocks >= 2LL * n_sms) return 0;
    return 2 * blocks >= 2LL * n_sms ? kStarletRows8 : kStarletRows4;
}

int launch_starlet(const FieldDev *fields, int n_fields, int Fmax, int forms, const ChunkItem *chunks,
                   int n_chunks, int Jmax, const float *params, double *l1_part, cudaStream_t st) {
    static std::once_flag configured;  // host threads evaluating at once configure the kernels once
    std::call_once(configured, [] {  // the band and tile kernels take their budgets of dynamic shared memory
        cudaFuncSetAttribute(starlet_band_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_band_adj_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_tile_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemBytes);
        cudaFuncSetAttribute(starlet_tile_adj_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemBytes);
        cudaFuncSetAttribute(starlet_band_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_band_adj_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_tile_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemBytes);
        cudaFuncSetAttribute(starlet_tile_adj_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemBytes);
        cudaFuncSetAttribute(starlet_comb_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_comb_adj_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_comb_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
        cudaFuncSetAttribute(starlet_comb_adj_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemBytes);
    });
    const bool bands = (forms & 1) != 0, tiles = (forms & 2) != 0;
    const bool combs = (forms & 8) != 0, map = (forms & kStarletMapBit) != 0;
    // comb bands: s combs of comb_chunks blocks at level j; staging of cr + 4 (forward) or
    // 2 cr + 4 (adjoint) rows of the widest comb-band grid
    const int cr = starlet_comb_rows_of(forms);
    const int Fc = std::min(Fmax, kCombMaxF);
    auto cgrid = [&](int j) { return dim3((unsigned)((1 << j) * comb_chunks(Fc, 1 << j, cr)), n_fields); };
    const int comb_fwd_smem = (cr + 4) * Fc * (int)sizeof(float);
    const int comb_adj_smem = (2 * cr + 4) * Fc * (int)sizeof(float);
    auto tgrid = [&](int j) {
        const int sj = 1 << j;
        return dim3((unsigned)(sj * comb_chunks(Fmax, sj) * ((Fmax + kTileCols - 1) / kTileCols)), n_fields);
    };
    auto tile_smem = [&](long long floats) {
        return (int)std::min<long long>(floats * (long long)sizeof(float), kTileSmemBytes);
    };
    int n = 0;
    const dim3 bgrid((Fmax + kBandRows - 1) / kBandRows, n_fields);
    // shared memory of level j: (2 * 16 + 4 * 2^j) rows of the widest grid, at most the budget
    // (which every banded field's deepest level fits, so its shallower levels fit too)
    auto band_smem = [&](int j) {
        const long long b = (2LL * kBandRows + 4LL * (1 << j)) * Fmax * (long long)sizeof(float);
        return (int)std::min<long long>(b, kBandSmemBytes);
    };
    for (int j = 0; j <= Jmax - 2; ++j) {
        if (bands) {
            if (map)
                starlet_band_fwd_kernel<true><<<bgrid, 256, band_smem(j), st>>>(fields, params, l1_part, j);
            else
                starlet_band_fwd_kernel<false><<<bgrid, 256, band_smem(j), st>>>(fields, params, l1_part, j);
            ++n;
        }
        if (combs) {
            if (map)
                starlet_comb_fwd_kernel<true><<<cgrid(j), 256, comb_fwd_smem, st>>>(fields, params, l1_part, j, cr);
            else
                starlet_comb_fwd_kernel<false><<<cgrid(j), 256, comb_fwd_smem, st>>>(fields, params, l1_part, j, cr);
            ++n;
        }
        if (tiles) {
            const int sm = tile_smem(tile_fwd_floats(j));
            if (map)
                starlet_tile_fwd_kernel<true><<<tgrid(j), 256, sm, st>>>(fields, params, l1_part, j);
            else
                starlet_tile_fwd_kernel<false><<<tgrid(j), 256, sm, st>>>(fields, params, l1_part, j);
            ++n;
        }
    }
    for (int j = Jmax - 2; j >= 0; --j) {
        if (bands) {
            if (map)
                starlet_band_adj_kernel<true><<<bgrid, 256, band_smem(j), st>>>(fields, params, j);
            else
                starlet_band_adj_kernel<false><<<bgrid, 256, band_smem(j), st>>>(fields, params, j);
            ++n;
        }
        if (combs) {
            if (map)
                starlet_comb_adj_kernel<true><<<cgrid(j), 256, comb_adj_smem, st>>>(fields, params, j, cr);
            else
                starlet_comb_adj_kernel<false><<<cgrid(j), 256, comb_adj_smem, st>>>(fields, params, j, cr);
            ++n;
        }
        if (tiles) {
            const int sm = tile_smem(tile_adj_floats(j));
            if (map)
                starlet_tile_adj_kernel<true><<<tgrid(j), 256, sm, st>>>(fields, params, j);
            else
                starlet_tile_adj_kernel<false><<<tgrid(j), 256, sm, st>>>(fields, params, j);
            ++n;
        }
    }
    return n;
}

}  // namespace sr
