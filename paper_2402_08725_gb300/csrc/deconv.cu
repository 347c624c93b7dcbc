// Joint multi-epoch deconvolution: loss and gradient kernels (sm_103a).
//
// The model of sec. 2.2 (Eq. 9-10) per epoch i is M_i = D S_i (h + P_i) + f^2 Gamma_i,
// with S_i the convolution by the narrow PSF s_i and D the f x f block sum.
// D is folded into S once per PSF (set_psfs):
//     M_i[p] = sum_u kappa_i(f p - u) f_i[u],   kappa_i(t) = sum_{a,b<f} s_i[t + (a,b) + o].
// Splitting the fine pixel u = f m + phi by its phase phi in [0,f)^2 turns this into f^2
// ordinary convolutions on the data grid:
//     M_i[p] = sum_phi sum_tau kappa_{i,phi}(tau) F_phi[p - tau],  F_phi[m] = f_i[f m + phi],
//     kappa_{i,phi}(tau) = kappa_i(f tau - phi),
// and the adjoint (D^T then S_i^T) becomes, per phase,
//     G_{i,phi}[m] = sum_tau kappa_{i,phi}(tau) e_i[m + tau],   e_i = -w (d_i - M_i).
// This needs f^2 times fewer multiply-adds than the fine-resolution form.
//
// Kernels here:
//   kappa_prep_kernel   folded polyphase kernels, once per set_psfs
//   fwd_kernel<R>       persistent over (field, epoch, tile): stage F_phi tiles of h plus the
//                       rasterised point sources in shared memory, accumulate M over all phases,
//                       residual, FP64 chi^2 and sum(e) partials (warp shuffles), write e
//   adj_kernel<R>       persistent over (field, epoch, tile): stage the e tile once, correlate
//                       with each phase's kernel, write G_{i,phi} (per-epoch images)
//   psgrad_kernel       per (epoch, source): <G_i, g>, <G_i, grad g> on the source window
//   hgrad_kernel        dL/dh = sum_i G_i + starlet prior gradient (fixed epoch order)
//   finalize_kernel     loss, dGamma, da, dc, ddelta per field in fixed order
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "corr.cuh"
#include "fold.cuh"
#include "reduce.cuh"

namespace sr {

// ---------------------------------------------------------------------------------------
// Folded kernels: kappa_{i,phi}(tau) for tau in [tau_lo, tau_lo + Tk)^2, stored
// [E][f*f][Tk][Tk] (phi = phy*f + phx).
// ---------------------------------------------------------------------------------------
__global__ void kappa_prep_kernel(const float *__restrict__ s, float *__restrict__ kappa, int E, int K, int f,
                                  int Tk, int tau_lo) {
    const long long per = (long long)f * f * Tk * Tk, total = (long long)E * per;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / per;
        kappa[idx] = kappa_fold(s + i * K * K, K, f, Tk, tau_lo, idx - i * per);
    }
}

void launch_kappa_prep(const float *s, float *kappa, int E, int K, int f, int Tk, int tau_lo, cudaStream_t st) {
    const long long total = (long long)E * f * f * Tk * Tk;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    kappa_prep_kernel<<<grid, 256, 0, st>>>(s, kappa, E, K, f, Tk, tau_lo);
}

struct TileGeom {
    int h, w, PG, per_group, g, row, chunk, xrows, xcols, xpitch, kpitch;
};

template <int R>
__device__ __forceinline__ TileGeom tile_geom(const TileItem &t, int Tk) {
    TileGeom G;
    G.h = t.h;
    G.w = t.w;
    G.PG = t.pg;
    const int chunks = G.w / R;
    G.per_group = G.h * chunks;
    G.g = threadIdx.x / G.per_group;
    const int l = threadIdx.x - G.g * G.per_group;
    G.row = l % G.h;       // consecutive lanes take consecutive rows: odd pitch -> no bank conflicts
    G.chunk = l / G.h;
    G.xrows = G.h + Tk - 1;
    G.xcols = G.w + Tk - 1;
    G.xpitch = (G.w + Tk) | 1;
    G.kpitch = (Tk + 3) & ~3;
    return G;
}

__device__ __forceinline__ int align4(int n) { return (n + 3) & ~3; }

// ceil(a / b) for b > 0 and any sign of a
__device__ __forceinline__ int ceil_div(int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); }

// Position of point source k in epoch i's frame: R_i c_k in a rotated frame, else c_k.
__device__ __forceinline__ float2 frame_pos(const FieldDev &fd, const float *__restrict__ c, int k, int i) {
    const float cx = c[2 * k], cy = c[2 * k + 1];
    if (!fd.rot) return make_float2(cx, cy);
    const float2 r = fd.rot[i];
    return make_float2(r.x * cx - r.y * cy, r.y * cx + r.x * cy);
}

// Fine-grid centre of a point source at frame position p in epoch i: (F-1)/2 + f (p + delta_i).
__device__ __forceinline__ float2 source_centre(float2 p, const float *__restrict__ dl, int F, int f) {
    const float u0 = 0.5f * (float)(F - 1);
    return make_float2(u0 + (float)f * (p.x + dl[0]), u0 + (float)f * (p.y + dl[1]));
}

// Bilinear value of h (F x F, zero outside) at the reference-frame point q, and its cell.
__device__ __forceinline__ float bilinear_h(const float *__restrict__ h, int F, float2 q) {
    const float fx = floorf(q.x), fy = floorf(q.y);
    const int x0 = (int)fx, y0 = (int)fy;
    const float tx = q.x - fx, ty = q.y - fy;
    float v = 0.f;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int yy = y0 + b;
        if (yy < 0 || yy >= F) continue;
        const float wy = b ? ty : 1.f - ty;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int xx = x0 + a;
            if (xx < 0 || xx >= F) continue;
            v += wy * (a ? tx : 1.f - tx) * __ldg(h + (long long)yy * F + xx);
        }
    }
    return v;
}

// Point sources are added while the tile is staged, each pixel summing the sources whose window
// holds it in index order (a fixed order for any M: the result does not depend on the schedule).
constexpr int kStagedSources = 64;  // the most point sources a problem may have

__device__ __forceinline__ float gauss_at(float dx, float dy) {
    return kGaussNorm * exp2f(-(dx * dx + dy * dy));
}

template <int R>
__global__ void __launch_bounds__(kThreads, 2)
fwd_kernel(const FieldDev *__restrict__ fields, const TileItem *__restrict__ items, int n_items,
           int *__restrict__ counter, const float *__restrict__ params, float *__restrict__ ebuf,
           double *__restrict__ chi_part, double *__restrict__ se_part) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_item;
    __shared__ float2 s_red[2][kThreads / 32];
    __shared__ float4 s_src[kStagedSources];
    __shared__ int2 s_win[kStagedSources];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const TileItem t = items[it];
        const FieldDev &fd = fields[t.field];
        const int f = fd.f, N = fd.N, F = fd.F, Tk = fd.Tk, M = fd.M, E = fd.E;
        const int thi = fd.tau_lo + Tk - 1;
        const int nph = f * f;
        const TileGeom G = tile_geom<R>(t, Tk);
        const int xsize = G.xrows * G.xpitch;
        float *Kall = smem + align4(G.PG * xsize);
        const float *hpar = params + fd.param_off;
        const float *apar = hpar + (long long)F * F + (long long)t.epoch * M;
        const float *cpar = hpar + (long long)F * F + (long long)E * M;
        const float *dpar = cpar + 2 * M + 2 * t.epoch;
        const float gam = cpar[2 * M + 2 * E + t.epoch];
        const int my0 = t.y0 - thi, mx0 = t.x0 - thi;  // data-grid origin of the staged tiles
        // the moved channel (translate): output fine pixel u reads h bilinearly at u + n + (0 | 1)
        int snx = 0, sny = 0;
        float stx = 0.f, sty = 0.f;
        if (fd.translate) {
            shift_split((float)f * dpar[0], &snx, &stx);
            shift_split((float)f * dpar[1], &sny, &sty);
        }
        // a rotated frame reads h bilinearly at frame_point(u) instead
        const float2 rcs = fd.rot ? fd.rot[t.epoch] : make_float2(1.f, 0.f);
        const float2 rsh = fd.translate ? make_float2((float)f * dpar[0], (float)f * dpar[1]) : make_float2(0.f, 0.f);

        // point sources of this epoch: fine centre, amplitude and window origin (Eq. 9)
        if (tid < M) {
            const float2 pos = frame_pos(fd, cpar, tid, t.epoch);
            const float2 cen = source_centre(pos, dpar, F, f);
            s_src[tid] = make_float4(pos.x, pos.y, apar[tid], 0.f);
            s_win[tid] = make_int2((int)floorf(cen.x) - kWinLo, (int)floorf(cen.y) - kWinLo);
        }
        __syncthreads();
        const int warp = tid >> 5, lane = tid & 31;

        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.f;

        for (int iter = 0; iter < nph / G.PG; ++iter) {
            // stage F_phi = f_i[f m + phi] = h + point sources (zero outside the grid), one row per warp
            for (int rr = warp; rr < G.PG * G.xrows; rr += kThreads / 32) {
                const int grp = rr / G.xrows;
                const int i = rr - grp * G.xrows;
                const int ph = iter * G.PG + grp;
                const int phy = ph / f, phx = ph - phy * f;
                const int my = my0 + i;
                float *dst = smem + grp * xsize + i * G.xpitch;
                if (my < 0 || my >= N) {
                    for (int j = lane; j < G.xcols; j += 32) dst[j] = 0.f;
                    continue;
                }
                const int uy = f * my + phy;
                // sources whose window holds this row: two ballots over the (at most 64) windows
                const bool in0 = lane < M && (unsigned)(uy - s_win[lane].y) < (unsigned)kWin;
                const bool in1 = lane + 32 < M && (unsigned)(uy - s_win[lane + 32].y) < (unsigned)kWin;
                const unsigned long long rowmask =
                    (unsigned long long)__ballot_sync(0xffffffffu, in0) |
                    ((unsigned long long)__ballot_sync(0xffffffffu, in1) << 32);
                const float *src = hpar + (long long)uy * F + phx;
                for (int j = lane; j < G.xcols; j += 32) {
                    const int mx = mx0 + j;
                    float v = 0.f;
                    if (mx >= 0 && mx < N) {
                        const int ux = f * mx + phx;
                        if (fd.rot) {
                            v = bilinear_h(hpar, F, frame_point(F, rcs, rsh, ux, uy));
                        } else if (fd.translate) {
                            // bilinear read at u - s, zero outside the grid
                            v = 0.f;
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                const int yy = uy + sny + b;
                                if (yy < 0 || yy >= F) continue;
                                const float wy = b ? sty : 1.f - sty;
#pragma unroll
                                for (int a = 0; a < 2; ++a) {
                                    const int xx = ux + snx + a;
                                    if (xx < 0 || xx >= F) continue;
                                    v += wy * (a ? stx : 1.f - stx) * __ldg(hpar + (long long)yy * F + xx);
                                }
                            }
                        } else {
                            v = __ldg(src + f * mx);
                        }
                        for (unsigned long long m = rowmask; m; m &= m - 1) {
                            const int k = __ffsll((long long)m) - 1;
                            if ((unsigned)(ux - s_win[k].x) < (unsigned)kWin)
                                v += s_src[k].z * gauss_at(src_offset(ux, F, f, s_src[k].x, dpar[0]),
                                                           src_offset(uy, F, f, s_src[k].y, dpar[1]));
                        }
                    }
                    dst[j] = v;
                }
            }
            // flipped folded kernels: Kp[jy][jx] = kappa_phi(thi - jy, thi - jx), one row per warp
            const int ksz = Tk * G.kpitch;
            const float *kap = fd.kappa + (long long)t.epoch * nph * Tk * Tk;
            for (int rr = warp; rr < G.PG * Tk; rr += kThreads / 32) {
                const int grp = rr / Tk;
                const int jy = rr - grp * Tk;
                const int ph = iter * G.PG + grp;
                const float *srow = kap + ((long long)ph * Tk + (Tk - 1 - jy)) * Tk + (Tk - 1);
                float *dst = Kall + grp * ksz + jy * G.kpitch;
                for (int jx = lane; jx < G.kpitch; jx += 32) dst[jx] = jx < Tk ? __ldg(srow - jx) : 0.f;
            }
            __syncthreads();
            if (G.g < G.PG)
                corr_accumulate<R>(acc, smem + G.g * xsize + G.row * G.xpitch + G.chunk * R, G.xpitch,
                                   Kall + G.g * ksz, G.kpitch, Tk);
            __syncthreads();
        }
        // sum the phase groups (fixed order)
        if (G.PG > 1) {
            float *red = smem;
            if (G.g >= 1 && G.g < G.PG) {
#pragma unroll
                for (int r = 0; r < R; ++r) red[((G.g - 1) * G.h + G.row) * G.w + G.chunk * R + r] = acc[r];
            }
            __syncthreads();
            if (G.g == 0) {
                for (int gg = 1; gg < G.PG; ++gg) {
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] += red[((gg - 1) * G.h + G.row) * G.w + G.chunk * R + r];
                }
            }
        }
        // residual, chi^2 and sum e (FP32 over the thread's R pixels, compensated across the
        // block), e = -w r
        float chi_r = 0.f, se_r = 0.f;
        const int py = t.y0 + G.row;
        if (G.g == 0 && py < N) {
            const float bg = (float)(f * f) * gam;
            const long long base = ((long long)t.epoch * N + py) * N;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int px = t.x0 + G.chunk * R + r;
                if (px < N) {
                    const float Mv = acc[r] + bg;
                    const float res = __ldg(fd.d + base + px) - Mv;
                    const float wv = __ldg(fd.w + base + px);
                    chi_r += 0.5f * wv * res * res;
                    const float e = -wv * res;
                    ebuf[fd.ebuf_off + base + px] = e;
                    se_r += e;
                }
            }
        }
        double chi = 0.0, se = 0.0;
        block_fsum2(FSum{chi_r, 0.f}, FSum{se_r, 0.f}, s_red, chi, se);
        if (tid == 0) {
            chi_part[t.slot] = chi;
            se_part[t.slot] = se;
        }
        __syncthreads();
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads)
adj_kernel(const FieldDev *__restrict__ fields, const TileItem *__restrict__ items, int n_items,
           int *__restrict__ counter, const float *__restrict__ ebuf, float *__restrict__ gbuf) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const TileItem t = items[it];
        const FieldDev &fd = fields[t.field];
        const int f = fd.f, N = fd.N, Tk = fd.Tk, tlo = fd.tau_lo;
        const int nph = f * f;
        const TileGeom G = tile_geom<R>(t, Tk);
        const int ysize = G.xrows * G.xpitch;
        float *Kall = smem + align4(ysize);
        const int my0 = t.y0 + tlo, mx0 = t.x0 + tlo;
        const float *ep = ebuf + fd.ebuf_off + (long long)t.epoch * N * N;
        // stage e on the tile plus halo (zero outside the data grid), one row per warp
        const int warp = tid >> 5, lane = tid & 31;
        for (int i = warp; i < G.xrows; i += kThreads / 32) {
            const int my = my0 + i;
            float *dst = smem + i * G.xpitch;
            const bool row_in = my >= 0 && my < N;
            const float *src = ep + (long long)my * N;
            for (int j = lane; j < G.xcols; j += 32) {
                const int mx = mx0 + j;
                dst[j] = (row_in && mx >= 0 && mx < N) ? src[mx] : 0.f;
            }
        }
        const int ksz = Tk * G.kpitch;
        const float *kap = fd.kappa + (long long)t.epoch * nph * Tk * Tk;
        float *gout = gbuf + fd.gbuf_off + (long long)t.epoch * nph * N * N;
        for (int iter = 0; iter < nph / G.PG; ++iter) {
            for (int rr = warp; rr < G.PG * Tk; rr += kThreads / 32) {
                const int grp = rr / Tk;
                const int jy = rr - grp * Tk;
                const int ph = iter * G.PG + grp;
                const float *srow = kap + ((long long)ph * Tk + jy) * Tk;
                float *dst = Kall + grp * ksz + jy * G.kpitch;
                for (int jx = lane; jx < G.kpitch; jx += 32) dst[jx] = jx < Tk ? __ldg(srow + jx) : 0.f;
            }
            __syncthreads();
            if (G.g < G.PG) {
                float acc[R];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = 0.f;
                corr_accumulate<R>(acc, smem + G.row * G.xpitch + G.chunk * R, G.xpitch, Kall + G.g * ksz,
                                   G.kpitch, Tk);
                const int ph = iter * G.PG + G.g;
                const int py = t.y0 + G.row;
                if (py < N) {
                    float *go = gout + ((long long)ph * N + py) * N;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int px = t.x0 + G.chunk * R + r;
                        if (px < N) go[px] = acc[r];
                    }
                }
            }
            __syncthreads();
        }
    }
}

// dL/da_ki = <G_i, g_ki>,  dL/d(centre) = a_ki <G_i, g_ki (u - centre)/sigma^2>  (window).
// One warp per (epoch, source) slot; ps_items[s] = (field, epoch, k).
__global__ void psgrad_kernel(const FieldDev *__restrict__ fields, const int4 *__restrict__ ps_items, int n,
                              const float *__restrict__ params, const float *__restrict__ gbuf,
                              float *__restrict__ ps_da, float *__restrict__ ps_du) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int4 w4 = ps_items[warp];
    const FieldDev &fd = fields[w4.x];
    const int i = w4.y, k = w4.z;
    const int f = fd.f, N = fd.N, F = fd.F, M = fd.M, E = fd.E;
    const int nph = f * f;
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
    const float *dpar = cpar + 2 * M + 2 * i;
    const float a = hpar[(long long)F * F + (long long)i * M + k];
    const float2 pos = frame_pos(fd, cpar, k, i);
    const float2 cen = source_centre(pos, dpar, F, f);
    const int uy_lo = (int)floorf(cen.y) - kWinLo, ux_lo = (int)floorf(cen.x) - kWinLo;
    const float *G = gbuf + fd.gbuf_off + (long long)i * nph * N * N;
    float sa = 0.f, sx = 0.f, sy = 0.f;
    for (int idx = lane; idx < kWin * kWin; idx += 32) {
        const int uy = uy_lo + idx / kWin, ux = ux_lo + idx % kWin;
        if (uy < 0 || uy >= F || ux < 0 || ux >= F) continue;
        const int my = uy / f, mx = ux / f;
        const int ph = (uy - my * f) * f + (ux - mx * f);
        const float gv = G[((long long)ph * N + my) * N + mx];
        const float dx = src_offset(ux, F, f, pos.x, dpar[0]);
        const float dy = src_offset(uy, F, f, pos.y, dpar[1]);
        const float gg = gv * gauss_at(dx, dy);
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
        const long long s = fd.ps_slot + (long long)i * M + k;
        ps_da[s] = sa;
        ps_du[2 * s] = a * kGaussInvSig2 * sx;
        ps_du[2 * s + 1] = a * kGaussInvSig2 * sy;
    }
}

// dL/dh[u] = T0[u] + sum_i G_i[u]: one thread per polyphase index q = phi*N*N + m.
__global__ void hgrad_kernel(const FieldDev *__restrict__ fields, const ChunkItem *__restrict__ chunks, int n_chunks,
                             const float *__restrict__ gbuf, float *__restrict__ grad, const float *__restrict__ params) {
    const int c = blockIdx.x;
    if (c >= n_chunks) return;
    const ChunkItem ch = chunks[c];
    const FieldDev &fd = fields[ch.field];
    if (fd.mode != 0) return;  // fields in the frequency-domain form get dL/dh from fft_hgrad_kernel
    const int q = ch.start + threadIdx.x;
    const int f = fd.f, N = fd.N, F = fd.F;
    if (q >= F * F) return;
    const long long plane = (long long)f * f * N * N;
    if (fd.rot) {
        // dL/dh = sum_i W_i^T G_i: pixel v gathers every u whose bilinear read (frame_point) has v
        // in its cell; those u lie within 1.5 pixels of u0 + s + R (v - u0) on each axis
        const int ph = q / (N * N), m = q - ph * N * N;
        const int vy = f * (m / N) + ph / f, vx = f * (m % N) + ph % f;
        const float *cpar = params + fd.param_off + (long long)F * F + (long long)fd.E * fd.M + 2 * fd.M;
        const float *Gb = gbuf + fd.gbuf_off;
        const float u0 = 0.5f * (float)(F - 1);
        float acc = 0.f;
        for (int i = 0; i < fd.E; ++i) {
            const float2 cs = fd.rot[i];
            const float2 sh = fd.translate ? make_float2((float)f * cpar[2 * i], (float)f * cpar[2 * i + 1])
                                           : make_float2(0.f, 0.f);
            const float ex = (float)vx - u0, ey = (float)vy - u0;
            const float cx = u0 + sh.x + (cs.x * ex - cs.y * ey), cy = u0 + sh.y + (cs.y * ex + cs.x * ey);
            const int ux0 = max(0, (int)ceilf(cx - 1.5f)), ux1 = min(F - 1, (int)floorf(cx + 1.5f));
            const int uy0 = max(0, (int)ceilf(cy - 1.5f)), uy1 = min(F - 1, (int)floorf(cy + 1.5f));
            float gi = 0.f;
            for (int uy = uy0; uy <= uy1; ++uy)
                for (int ux = ux0; ux <= ux1; ++ux) {
                    const float2 qp = frame_point(F, cs, sh, ux, uy);
                    const float fx = floorf(qp.x), fy = floorf(qp.y);
                    const int a = vx - (int)fx, b = vy - (int)fy;
                    if ((unsigned)a > 1u || (unsigned)b > 1u) continue;
                    const float tx = qp.x - fx, ty = qp.y - fy;
                    const int uph = (uy % f) * f + ux % f;
                    gi += (b ? ty : 1.f - ty) * (a ? tx : 1.f - tx) *
                          Gb[(long long)i * plane + (long long)uph * N * N + (uy / f) * N + ux / f];
                }
            acc += gi;
        }
        const int u = vy * F + vx;
        grad[fd.param_off + u] = acc + fd.starlet[(long long)fd.J * F * F + u];
        return;
    }
    if (fd.translate) {
        // dL/dh = sum_i T_i^T G_i: pixel v gathers G_i(v - n - (0 | 1)) with the read's weights
        const int ph = q / (N * N), m = q - ph * N * N;
        const int vy = f * (m / N) + ph / f, vx = f * (m % N) + ph % f;
        const float *cpar = params + fd.param_off + (long long)F * F + (long long)fd.E * fd.M + 2 * fd.M;
        const float *Gb = gbuf + fd.gbuf_off;
        float acc = 0.f;
        for (int i = 0; i < fd.E; ++i) {
            int nx, ny;
            float tx, ty;
            shift_split((float)f * cpar[2 * i], &nx, &tx);
            shift_split((float)f * cpar[2 * i + 1], &ny, &ty);
            float gi = 0.f;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int uy = vy - ny - b;
                if (uy < 0 || uy >= F) continue;
                const float wy = b ? ty : 1.f - ty;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ux = vx - nx - a;
                    if (ux < 0 || ux >= F) continue;
                    const int uph = (uy % f) * f + ux % f;
                    gi += wy * (a ? tx : 1.f - tx) *
                          Gb[(long long)i * plane + (long long)uph * N * N + (uy / f) * N + ux / f];
                }
            }
            acc += gi;
        }
        const int u = vy * F + vx;
        grad[fd.param_off + u] = acc + fd.starlet[(long long)fd.J * F * F + u];
        return;
    }
    const float *G = gbuf + fd.gbuf_off + q;
    // four interleaved FP32 partial sums over the epochs, combined in a fixed order
    // (the FP64 pipe of this GPU is far narrower than the FP32 one)
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int i = 0;
    for (; i + 4 <= fd.E; i += 4) {
        s0 += G[(long long)i * plane];
        s1 += G[(long long)(i + 1) * plane];
        s2 += G[(long long)(i + 2) * plane];
        s3 += G[(long long)(i + 3) * plane];
    }
    for (; i < fd.E; ++i) s0 += G[(long long)i * plane];
    const int ph = q / (N * N), m = q - ph * N * N;
    const int my = m / N, mx = m - my * N;
    const int u = (f * my + ph / f) * F + f * mx + ph % f;
    const float *T0 = fd.starlet + (long long)fd.J * F * F;
    grad[fd.param_off + u] = ((s0 + s1) + (s2 + s3)) + T0[u];
}

// The moved channel's part of dL/d delta_i = f sum_u G_i(u) d(T h)(u)/d s, with d(T h)/d s_x =
// -[(1 - t_y)(h(y0, x0 + 1) - h(y0, x0)) + t_y (h(y0 + 1, x0 + 1) - h(y0 + 1, x0))] (and the same with
// the axes swapped), (x0, y0) = u + n.  Block (epoch, field); compensated FP32 sums in fixed order.
__global__ void __launch_bounds__(256)
hshift_grad_kernel(const FieldDev *__restrict__ fields, const float *__restrict__ params,
                   const float *__restrict__ gbuf, float *__restrict__ hs) {
    __shared__ float4 s_red[8];
    const FieldDev &fd = fields[blockIdx.y];
    const int i = blockIdx.x;
    if (!fd.translate || fd.mode != 0 || i >= fd.E) return;
    const int f = fd.f, N = fd.N, F = fd.F;
    const float *h = params + fd.param_off;
    const float *cpar = h + (long long)F * F + (long long)fd.E * fd.M + 2 * fd.M;
    int nx, ny;
    float tx, ty;
    shift_split((float)f * cpar[2 * i], &nx, &tx);
    shift_split((float)f * cpar[2 * i + 1], &ny, &ty);
    const float *Gi = gbuf + fd.gbuf_off + (long long)i * f * f * N * N;
    auto hv = [&](int y, int x) { return (y < 0 || y >= F || x < 0 || x >= F) ? 0.f : h[(long long)y * F + x]; };
    const float2 cs = fd.rot ? fd.rot[i] : make_float2(1.f, 0.f);
    const float2 sh = make_float2((float)f * cpar[2 * i], (float)f * cpar[2 * i + 1]);
    FSum sx = fsum_zero(), sy = fsum_zero();
    for (int q = threadIdx.x; q < F * F; q += blockDim.x) {
        const int ph = q / (N * N), m = q - ph * N * N;
        const int uy = f * (m / N) + ph / f, ux = f * (m % N) + ph % f;
        const float G = Gi[q];
        int x0 = ux + nx, y0 = uy + ny;
        float wx = tx, wy = ty;
        if (fd.rot) {  // the cell of frame_point(u); d out / d s = -R grad H
            const float2 qp = frame_point(F, cs, sh, ux, uy);
            const float fx = floorf(qp.x), fy = floorf(qp.y);
            x0 = (int)fx;
            y0 = (int)fy;
            wx = qp.x - fx;
            wy = qp.y - fy;
        }
        const float h00 = hv(y0, x0), h01 = hv(y0, x0 + 1), h10 = hv(y0 + 1, x0), h11 = hv(y0 + 1, x0 + 1);
        const float gx = (1.f - wy) * (h01 - h00) + wy * (h11 - h10);
        const float gy = (1.f - wx) * (h10 - h00) + wx * (h11 - h01);
        const float dx = -(cs.x * gx - cs.y * gy), dy = -(cs.y * gx + cs.x * gy);
        sx = fsum_add(sx, G * dx);
        sy = fsum_add(sy, G * dy);
    }
    sx = fsum_warp(sx);
    sy = fsum_warp(sy);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        FSum ax = fsum_zero(), ay = fsum_zero();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ax = fsum_add(ax, FSum{s_red[w].x, s_red[w].y});
            ay = fsum_add(ay, FSum{s_red[w].z, s_red[w].w});
        }
        hs[fd.hs_off + 2 * i] = (float)((double)f * fsum_value(ax));
        hs[fd.hs_off + 2 * i + 1] = (float)((double)f * fsum_value(ay));
    }
}

// Per-field assembly of the loss and the small parameter blocks, in fixed order.
__global__ void __launch_bounds__(kThreads)
finalize_kernel(const FieldDev *__restrict__ fields, const double *__restrict__ chi_part,
                const double *__restrict__ se_part, const double *__restrict__ l1_part,
                const float *__restrict__ ps_da, const float *__restrict__ ps_du, float *__restrict__ grad,
                double *__restrict__ losses, const FieldDev *__restrict__ pts_fields,
                const double *__restrict__ l1_pts, const float *__restrict__ pts_g, const float *__restrict__ hs) {
    __shared__ double s_red[2][kThreads / 32];
    const FieldDev &fd = fields[blockIdx.x];
    const int E = fd.E, M = fd.M, F = fd.F, f = fd.f;
    // point-source prior of the field (Eq. 11, third term), if it has one
    const FieldDev *sd = (pts_fields && fd.pts > 0) ? &pts_fields[fd.pts - 1] : nullptr;
    // four interleaved partial sums per thread (slot s into (s / blockDim) mod 4), combined in a
    // fixed order: wide grids have tens of thousands of prior partials per field, whose loads a
    // single dependent chain per thread would serialise
    const long long nt = (long long)E * fd.n_tiles;
    const long long nl = (long long)(fd.J - 1) * fd.n_chunks;
    double chi = strided_sum4(chi_part + fd.tile_slot, nt);
    double l1 = strided_sum4(l1_part + fd.l1_slot, nl);
    if (sd) l1 += strided_sum4(l1_pts + sd->l1_slot, nl);
    block_sum2(chi, l1, s_red);
    if (threadIdx.x == 0) losses[blockIdx.x] = chi + l1;
    float *g = grad + fd.param_off + (long long)F * F;  // a block
    for (int s = threadIdx.x; s < E * M; s += blockDim.x)
        g[s] = sd ? ps_da[fd.ps_slot + s] + pts_g[3 * (sd->ps_slot + s % M)] / (float)E : ps_da[fd.ps_slot + s];
    float *gc = g + (long long)E * M;
    // d/dc_k sums over the epochs: one warp per (source, axis), lanes striding the epochs, then a
    // fixed shuffle tree (many epochs per field keep their loads in flight together)
    {
        const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
        for (int s = threadIdx.x >> 5; s < 2 * M; s += nwarp) {
            const int k = s >> 1, ax = s & 1;
            double acc = 0.0;
            if (fd.rot) {  // the centre is u0 + f (R_i c_k + delta_i): d/dc_k = f sum_i R_i^T d/d(centre)
                for (int i = lane; i < E; i += 32) {
                    const float2 r = fd.rot[i];
                    const long long b = 2 * (fd.ps_slot + (long long)i * M + k);
                    const double gx = ps_du[b], gy = ps_du[b + 1];
                    acc += ax == 0 ? (double)r.x * gx + (double)r.y * gy : -(double)r.y * gx + (double)r.x * gy;
                }
            } else {
                for (int i = lane; i < E; i += 32) acc += (double)ps_du[2 * (fd.ps_slot + (long long)i * M + k) + ax];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0)
                gc[s] = sd ? (float)(f * acc + (double)pts_g[3 * (sd->ps_slot + k) + 1 + ax]) : (float)(f * acc);
        }
    }
    float *gd = gc + 2 * M;
    // d/ddelta_i: the epoch's sources in four interleaved partial sums (k mod 4, each in increasing
    // k), combined in a fixed order, so that a thread's loads are in flight together
    for (int s = threadIdx.x; s < 2 * E; s += blockDim.x) {
        const int i = s >> 1, ax = s & 1;
        const float *pu = ps_du + 2 * (fd.ps_slot + (long long)i * M) + ax;
        double p[4] = {0.0, 0.0, 0.0, 0.0};
        int k = 0;
        for (; k + 4 <= M; k += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] += (double)pu[2 * (k + u)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (k + u < M) p[u] += (double)pu[2 * (k + u)];
        const double acc = (p[0] + p[1]) + (p[2] + p[3]);
        gd[s] = (float)(f * acc) + ((hs && fd.translate) ? hs[fd.hs_off + s] : 0.f);
    }
    float *gg = gd + 2 * E;
    // dGamma_i = f^2 sum over the epoch's tiles: one thread per epoch for a few tiles per epoch;
    // one warp per epoch (lanes stride the tiles, then a fixed shuffle tree) for many, so that
    // their loads are in flight together
    if (fd.n_tiles <= 32) {
        for (int i = threadIdx.x; i < E; i += blockDim.x) {
            const double *sp = se_part + fd.tile_slot + (long long)i * fd.n_tiles;
            double p[4] = {0.0, 0.0, 0.0, 0.0};
            int tt = 0;
            for (; tt + 4 <= fd.n_tiles; tt += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) p[u] += sp[tt + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (tt + u < fd.n_tiles) p[u] += sp[tt + u];
            gg[i] = (float)((double)(f * f) * ((p[0] + p[1]) + (p[2] + p[3])));
        }
        return;
    }
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < E; i += nwarp) {
        double acc = 0.0;
        const double *sp = se_part + fd.tile_slot + (long long)i * fd.n_tiles;
        for (int tt = lane; tt < fd.n_tiles; tt += 32) acc += sp[tt];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) gg[i] = (float)((double)(f * f) * acc);
    }
}

__global__ void total_kernel(const double *__restrict__ losses, int n, double *__restrict__ total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += losses[i];
        *total = s;
    }
}

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
static int fwd_smem_bytes_item(const TileItem &t, int Tk, bool fwd) {
    const int xrows = t.h + Tk - 1;
    const int xpitch = (t.w + Tk) | 1;
    const int kpitch = (Tk + 3) & ~3;
    const int xs = fwd ? t.pg * xrows * xpitch : xrows * xpitch;
    int red = 0;
    if (fwd && t.pg > 1) red = (t.pg - 1) * t.h * t.w;
    int xpart = ((xs + 3) & ~3);
    if (red > xpart) xpart = (red + 3) & ~3;
    return (xpart + t.pg * Tk * kpitch) * (int)sizeof(float);
}

int tile_smem_bytes(const TileItem &t, int Tk, bool fwd) { return fwd_smem_bytes_item(t, Tk, fwd); }

// The most phase groups (a divisor of f^2) whose threads fit in one block and whose forward
// tile fits in smem_limit bytes of shared memory; 1 if none does.
int choose_tile_pg(int nph, TileItem t, int Tk, int smem_limit) {
    int best = 1;
    const int threads_per_group = t.h * (t.w / kR);
    for (int pg = 1; pg <= nph; ++pg) {
        if (nph % pg != 0 || pg * threads_per_group > kThreads) continue;
        t.pg = pg;
        if (tile_smem_bytes(t, Tk, true) > smem_limit) continue;
        best = pg;
    }
    return best;
}

sr_status configure_tile_kernels(int smem_fwd, int smem_adj) {
    SR_CUDA(cudaFuncSetAttribute(fwd_kernel<kR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_fwd));
    SR_CUDA(cudaFuncSetAttribute(adj_kernel<kR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_adj));
    return SR_OK;
}

sr_status occupancy_tile_kernels(int smem_fwd, int smem_adj, int *blocks_fwd, int *blocks_adj) {
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_fwd, fwd_kernel<kR>, kThreads, smem_fwd));
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_adj, adj_kernel<kR>, kThreads, smem_adj));
    return SR_OK;
}

void launch_fwd(const FieldDev *fields, const TileItem *items, int n_items, int *counter, const float *params,
                float *ebuf, double *chi_part, double *se_part, int grid, int smem, cudaStream_t st) {
    fwd_kernel<kR><<<grid, kThreads, smem, st>>>(fields, items, n_items, counter, params, ebuf, chi_part, se_part);
}

void launch_adj(const FieldDev *fields, const TileItem *items, int n_items, int *counter, const float *ebuf,
                float *gbuf, int grid, int smem, cudaStream_t st) {
    adj_kernel<kR><<<grid, kThreads, smem, st>>>(fields, items, n_items, counter, ebuf, gbuf);
}

void launch_psgrad(const FieldDev *fields, const int4 *ps_items, int n, const float *params, const float *gbuf,
                   float *ps_da, float *ps_du, cudaStream_t st) {
    if (n <= 0) return;
    const int warps_per_block = 8;
    psgrad_kernel<<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        fields, ps_items, n, params, gbuf, ps_da, ps_du);
}

void launch_hgrad(const FieldDev *fields, const ChunkItem *chunks, int n_chunks, const float *gbuf, float *grad,
                  const float *params, cudaStream_t st) {
    hgrad_kernel<<<n_chunks, 256, 0, st>>>(fields, chunks, n_chunks, gbuf, grad, params);
}

void launch_hshift_grad(const FieldDev *fields, int n_fields, int E_max, const float *params, const float *gbuf,
                        float *hs, cudaStream_t st) {
    hshift_grad_kernel<<<dim3(E_max, n_fields), 256, 0, st>>>(fields, params, gbuf, hs);
}

void launch_finalize(const FieldDev *fields, int n_fields, const double *chi_part, const double *se_part,
                     const double *l1_part, const float *ps_da, const float *ps_du, float *grad, double *losses,
                     double *total, cudaStream_t st, const FieldDev *pts_fields, const double *l1_pts,
                     const float *pts_g, const float *hs) {
    finalize_kernel<<<n_fields, kThreads, 0, st>>>(fields, chi_part, se_part, l1_part, ps_da, ps_du, grad, losses,
                                                   pts_fields, l1_pts, pts_g, hs);
    total_kernel<<<1, 32, 0, st>>>(losses, n_fields, total);
}

}  // namespace sr
