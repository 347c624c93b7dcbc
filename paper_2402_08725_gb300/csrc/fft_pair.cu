// Frequency-domain form of the deconvolution loss and gradient: in-place transforms of real
// image pairs (sm_103a).
//
// The D-folded polyphase model is a sum over phases phi of data-grid convolutions,
// M_i = sum_phi kappa_{i,phi} * F_phi (Eq. 8-10 with the block sum folded into the kernels), and
// its adjoint a correlation per phase.  With circular transforms of size L x L,
// L >= N + max(tau_hi, -tau_lo), the wrap-around never reaches the N x N output, so
//     M_i = IDFT( sum_phi Khat_{i,phi} (Hhat_phi + Phat_{i,phi}) )          on [0,N)^2,
//     dL/dh_phi = IDFT( sum_i conj(Khat_{i,phi}) ehat_i )                   on [0,N)^2,
// exactly up to rounding.  Khat (spectra of the folded kernels) are computed at set_psfs, Hhat
// (the phase images of h) once per evaluation, the point sources' spectra are outer products of
// 1-D DFTs of the sampled Gaussian window, and their gradients come from Parseval's identity.
//
// Every transform here is a complex L x L transform of two real images at once (real and
// imaginary parts): two epochs of a chunk, or two phases of a field.  The half spectra of the two
// are separated (or joined) with Hermitian symmetry: X_a(k) = (Z(k) + conj Z(-k)) / 2,
// X_b(k) = (Z(k) - conj Z(-k)) / (2i), and Z = X_a + i X_b.  A length-L transform, L = R1 R2, is
// two passes of in-register DFTs that read and write the same shared-memory positions (so one
// buffer per pair and no barrier inside a pass):
//   pass A: for each n2 < R2, the R1-point DFT over n1 of x[n2 + R2 n1], times W_L^(n2 k1),
//           written back to positions n2 + R2 k1;
//   pass B: for each k1 < R1, the R2-point DFT of the R2 consecutive values at R2 k1 + n2,
//           written back in place: X[k1 + R1 k2] lands at position R2 k1 + k2.
// Spectra therefore live in "digit-transposed" order on both axes (frequency k at position
// R2 (k mod R1) + k / R1); the inverse runs the passes backwards (B then A) from that order and
// returns the natural spatial order, so nothing is ever reordered.  Along x, every group of R2
// positions is padded to an odd length S (the stride of pass B and of the spectral loops across a
// warp), and rows have a pitch P = R2 (mod 16) where shared memory allows, so that the row passes
// and the spectral loops touch 16 different 8-byte slots per half-warp.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"
#include "ffsum.cuh"
#include "fft_pair.cuh"
#include "kernels.cuh"

namespace sr {
namespace {

// --- the per-epoch chunk kernel ---------------------------------------------------------------
struct PrShared {
    // the work item's parameters: amplitudes a_{i,k}, epoch shifts delta_i, backgrounds gamma_i of
    // its epochs, and the source positions c_k (loaded once per item)
    float ia[kFftChunk * kFftMaxSources];
    float id[2 * kFftChunk];
    float ig[kFftChunk];
    float ic[2 * kFftMaxSources];
    int item;
};
__shared__ PrShared pr_sh;

// profile tables: [epoch of the group][source][phase][kind][H], kind 0 gx, 1 d gx, 2 gy, 3 d gy
__device__ __forceinline__ int prof_at(int e, int k, int ph, int kind, int M, int f, int H) {
    return (((e * M + k) * f + ph) * 4 + kind) * H;
}

// One item (x = field, y = first epoch, z = end, w = chunk index within the field) in groups of GP
// epoch pairs; MS bounds the sources.  Not inlined: each variant is register-allocated on its own.
template <int L, int GP, int MS>
__device__ __noinline__ void chunk_item_pair(const FieldDev &fd, const int4 item, const float *__restrict__ params,
                                             const float2 *__restrict__ hhat_all, float2 *__restrict__ acc_all,
                                             double *__restrict__ chi_part, double *__restrict__ se_part,
                                             float *__restrict__ ps_da, float *__restrict__ ps_du) {
    using G = Pr<L>;
    constexpr int H = G::H, HP = G::HP, LHP = L * HP, ZN = G::ZN, P = G::P;
    constexpr int EG = 2 * GP;             // epochs per group
    constexpr int RS = GP == 1 ? 2 : 1;    // rows per thread and step of the model loop
    constexpr int PC = GP == 4 ? 2 : 4;    // phases whose model-loop loads are issued together
    constexpr int RA = GP == 1 ? 4 : GP == 2 ? 2 : 1;  // rows per thread and step of the adjoint loop
    constexpr int RP = kFftThreads / H;    // rows in parallel
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int f = fd.f, N = fd.N, F = fd.F, M = fd.M, E = fd.E, nph = f * f;
    PrShared &sh = pr_sh;
    float2 *Z = pr_dyn;
    float2 *prof = Z + GP * ZN;
    float2 *TWL = prof + EG * M * f * 4 * H;
    load_twl<L>(TWL, fd.fft_tw);
    const float *hpar = params + fd.param_off;
    const float *cpar = hpar + (long long)F * F + (long long)E * M;
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
    const int tx = tid % H, ty = tid / H;
    const int cx = kcol<L>(tx), cxm = kcol<L>(neg_mod(tx, L));
    const bool selfcol = tx == 0 || 2 * tx == L;   // columns whose conjugate partner is in the column
    const float wgt = selfcol ? 1.f : 2.f;          // Parseval weight of the column
    const unsigned long long pol_last = l2_policy_last(), pol_first = l2_policy_first();
    const int nv = 2 + 3 * M;                       // reduced values per epoch
    for (int i0 = item.y; i0 < item.z; i0 += EG) {
        const int ne = min(EG, item.z - i0);
        const int np = (ne + 1) / 2;
        const float2 *kh = fd.fft_khat + (long long)i0 * nph * LHP;  // [e][phi][L][HP]
        const float *apar = sh.ia + (i0 - item.y) * M;                 // a_{i0 + e, k} at e M + k
        // The next group's data and weights go to L2 while this one computes (sizes are multiples of
        // 16 bytes when N is even).  The kernel spectra are not prefetched: with every SM streaming
        // its own group's spectra, an early copy in L2 is evicted before its use (measured slower).
        if (tid == 0 && i0 + EG < item.z && (N & 1) == 0) {
            const int nn = min(EG, item.z - i0 - EG);
            prefetch_l2(fd.d + (long long)(i0 + EG) * N * N, (long long)nn * N * N * 4);
            prefetch_l2(fd.w + (long long)(i0 + EG) * N * N, (long long)nn * N * N * 4);
        }
        // 1-D DFTs (frequencies 0 .. L/2) of the window profiles g1(u - c) and g1(u - c) (u - c) / sigma^2
        // on each phase's sub-grid u = f m + phase
        {
            const int per = M * f * 2 * H;
            for (int idx = tid; idx < ne * per; idx += nt) {
                const int e = idx / per, rr = idx - e * per;
                const int kk = rr % H, q = rr / H;
                const int xy = q & 1, kf = q >> 1;
                const int k = kf / f, phs = kf - k * f;
                const float cpos = sh.ic[2 * k + xy], dl = sh.id[2 * (i0 - item.y + e) + xy];
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
                    const float2 w = __ldg(&fd.fft_tw[(kk * m) % L]);  // kk < L, 0 <= m <= N + 1
                    v.x += gv * w.x;
                    v.y += gv * w.y;
                    vd.x += gd * w.x;
                    vd.y += gd * w.y;
                }
                float2 *pt = prof + prof_at(e, k, phs, 2 * xy, M, f, H) + kk;
                pt[0] = v;
                pt[H] = vd;
            }
        }
        __syncthreads();
        // model spectra: M_e = sum_phi Khat_{e,phi} (Hhat_phi + sum_k a_{e,k} gx gy) on the half plane,
        // written as Z = M_{2g} + i M_{2g+1} at k and its conjugate at -k.  Every load of PC phases
        // of RS rows is issued before any is used (one round trip per PC phases).
        if (ty < RP) {
            for (int row0 = ty; row0 < L; row0 += RS * RP) {
                float2 m[RS][EG];
#pragma unroll
                for (int j = 0; j < RS; ++j)
#pragma unroll
                    for (int e = 0; e < EG; ++e) m[j][e] = make_float2(0.f, 0.f);
                for (int ph0 = 0; ph0 < nph; ph0 += PC) {
                    float2 hv[PC][RS], kv[PC][RS][EG];
#pragma unroll
                    for (int q = 0; q < PC; ++q) {
                        const int ph = ph0 + q;
#pragma unroll
                        for (int j = 0; j < RS; ++j) {
                            const int row = row0 + j * RP;
                            const bool ok = row < L && ph < nph;
                            const int off = ph * LHP + row * HP + tx;
                            hv[q][j] = ok ? ldg_hint(hh + off, pol_last) : make_float2(0.f, 0.f);
#pragma unroll
                            for (int e = 0; e < EG; ++e)
                                kv[q][j][e] = (ok && e < ne) ? ldg_hint(kh + e * nph * LHP + off, pol_last)
                                                             : make_float2(0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < PC; ++q) {
                        const int ph = ph0 + q;
                        if (ph >= nph) break;
                        const int phy = ph / f, phx = ph - phy * f;
                        // a_{e,k} gx(kx) of this column and phase, once for the thread's rows
                        float2 agx[EG][MS];
#pragma unroll
                        for (int e = 0; e < EG; ++e)
#pragma unroll
                            for (int k = 0; k < MS; ++k) {
                                agx[e][k] = make_float2(0.f, 0.f);
                                if (k < M && e < ne) {
                                    const float2 gx = prof[prof_at(e, k, phx, 0, M, f, H) + tx];
                                    const float a = apar[e * M + k];
                                    agx[e][k] = make_float2(a * gx.x, a * gx.y);
                                }
                            }
#pragma unroll
                        for (int j = 0; j < RS; ++j) {
                            const int row = row0 + j * RP;
                            const bool lowrow = 2 * row <= L;
                            const int yr = lowrow ? row : L - row;
#pragma unroll
                            for (int e = 0; e < EG; ++e) {
                                if (e < ne && row < L) {
                                    float2 sv = hv[q][j];
#pragma unroll
                                    for (int k = 0; k < MS; ++k) {
                                        if (k < M) {
                                            float2 gy = prof[prof_at(e, k, phy, 2, M, f, H) + yr];
                                            if (!lowrow) gy.y = -gy.y;
                                            sv = cadd(sv, cmul(agx[e][k], gy));
                                        }
                                    }
                                    m[j][e] = cadd(m[j][e], cmul(kv[q][j][e], sv));
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < RS; ++j) {
                    const int ky = row0 + j * RP;
                    if (ky >= L || (selfcol && 2 * ky > L)) continue;  // the partner thread writes both
                    const int r = krow<L>(ky), rm = krow<L>(neg_mod(ky, L));
                    const bool self = selfcol && (ky == 0 || 2 * ky == L);
#pragma unroll
                    for (int g = 0; g < GP; ++g) {
                        const float2 M0 = m[j][2 * g], M1 = m[j][2 * g + 1];
                        float2 *zg = Z + g * ZN;
                        if (self) {
                            zg[r * P + cx] = make_float2(M0.x, M1.x);
                        } else {
                            zg[r * P + cx] = make_float2(M0.x - M1.y, M0.y + M1.x);    // M0 + i M1
                            zg[rm * P + cxm] = make_float2(M0.x + M1.y, M1.x - M0.y);  // conj(M0) + i conj(M1)
                        }
                    }
                }
            }
        }
        __syncthreads();
        cols_inv<L>(Z, np, N, TWL);
        rows_inv<L>(Z, np, N, N, TWL);
        // residual on [0,N)^2 in place (e = -w r for the forward transform), chi^2 and sum e per
        // epoch: the warps w with w mod GP = g take the rows of pair g
        FSum chi[2], se[2];
        chi[0] = chi[1] = se[0] = se[1] = fsum_zero();
        {
            const int g = warp % GP, sub = warp / GP, nsub = nw / GP;
            const int e0 = 2 * g, e1 = e0 + 1;
            if (e0 < ne) {
                const bool has1 = e1 < ne;
                const int i = i0 + e0;
                const float bg0 = (float)(f * f) * sh.ig[i - item.y];
                const float bg1 = has1 ? (float)(f * f) * sh.ig[i + 1 - item.y] : 0.f;
                const float *d0 = fd.d + (long long)i * N * N, *w0 = fd.w + (long long)i * N * N;
                const float *d1 = d0 + N * N, *w1 = w0 + N * N;
                float2 *zg = Z + g * ZN;
                // two rows per iteration: 32 data and weight loads per lane in flight together
                for (int y0 = sub; y0 < N; y0 += 2 * nsub) {
                    float c0 = 0.f, c1 = 0.f, s0 = 0.f, s1 = 0.f;
                    for (int x0 = 0; x0 < N; x0 += 128) {
                        float dv[2][4][2], wv[2][4][2];
#pragma unroll
                        for (int ry = 0; ry < 2; ++ry) {
                            const int y = y0 + ry * nsub;
#pragma unroll
                            for (int jx = 0; jx < 4; ++jx) {
                                const int x = x0 + 32 * jx + lane;
                                const bool in = x < N && y < N;
                                const int o = y * N + x;
                                dv[ry][jx][0] = in ? ldg_hint(d0 + o, pol_first) : 0.f;
                                wv[ry][jx][0] = in ? ldg_hint(w0 + o, pol_first) : 0.f;
                                dv[ry][jx][1] = (in && has1) ? ldg_hint(d1 + o, pol_first) : 0.f;
                                wv[ry][jx][1] = (in && has1) ? ldg_hint(w1 + o, pol_first) : 0.f;
                            }
                        }
#pragma unroll
                        for (int ry = 0; ry < 2; ++ry) {
                            const int y = y0 + ry * nsub;
                            if (y >= N) continue;
#pragma unroll
                            for (int jx = 0; jx < 4; ++jx) {
                                const int x = x0 + 32 * jx + lane;
                                if (x < N) {
                                    float2 *zp = zg + y * P + pcol<L>(x);
                                    const float2 mv = *zp;
                                    const float r0 = dv[ry][jx][0] - (mv.x * scale + bg0);
                                    const float r1 = dv[ry][jx][1] - (mv.y * scale + bg1);
                                    c0 += 0.5f * wv[ry][jx][0] * r0 * r0;
                                    c1 += 0.5f * wv[ry][jx][1] * r1 * r1;
                                    const float ev0 = -wv[ry][jx][0] * r0, ev1 = has1 ? -wv[ry][jx][1] * r1 : 0.f;
                                    s0 += ev0;
                                    s1 += ev1;
                                    *zp = make_float2(ev0, ev1);
                                }
                            }
                        }
                    }
                    chi[0] = fsum_add(chi[0], c0);
                    chi[1] = fsum_add(chi[1], c1);
                    se[0] = fsum_add(se[0], s0);
                    se[1] = fsum_add(se[1], s1);
                }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                chi[q] = fsum_warp(chi[q]);
                se[q] = fsum_warp(se[q]);
            }
        }
        __syncthreads();
        rows_fwd<L>(Z, np, N, N, TWL);
        cols_fwd<L>(Z, np, N, TWL);
        // adjoint spectra: acc_phi += sum_e conj(Khat_{e,phi}) ehat_e (epochs in order), and the
        // sources' Parseval products (weight 1 at kx = 0 and L/2, 2 elsewhere)
        const bool first = i0 == item.y, last = i0 + EG >= item.z;
        float pa[EG][MS], px[EG][MS], py[EG][MS];
#pragma unroll
        for (int e = 0; e < EG; ++e)
#pragma unroll
            for (int k = 0; k < MS; ++k) pa[e][k] = px[e][k] = py[e][k] = 0.f;
        // Phases outermost: with the column kx of the thread fixed, the Parseval sums factor as
        // sum_rows w Re(G conj(gx gy)) = w Re(conj(gx) T1), T1 = sum_rows G conj(gy) (and T2 with the
        // derivative profile gyd), so per point only T1 and T2 are accumulated.
        if (ty < RP) {
            for (int ph = 0; ph < nph; ++ph) {
                const int phy = ph / f, phx = ph - phy * f;
                float2 T1[EG][MS], T2[EG][MS];
#pragma unroll
                for (int e = 0; e < EG; ++e)
#pragma unroll
                    for (int k = 0; k < MS; ++k) T1[e][k] = T2[e][k] = make_float2(0.f, 0.f);
                for (int row0 = ty; row0 < L; row0 += RA * RP) {
                    float2 eh[RA][EG], av[RA], kv[RA][EG];
#pragma unroll
                    for (int j = 0; j < RA; ++j) {
                        const int row = row0 + j * RP;
                        const bool ok = row < L;
                        const int off = ph * LHP + row * HP + tx;
                        av[j] = (ok && !first) ? ld_hint(acc + off, pol_last) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int e = 0; e < EG; ++e)
                            kv[j][e] = (ok && e < ne) ? ldg_hint(kh + e * nph * LHP + off, pol_first)
                                                      : make_float2(0.f, 0.f);
                        const int ky = ok ? row : 0;
                        const int r = krow<L>(ky), rm = krow<L>(neg_mod(ky, L));
#pragma unroll
                        for (int g = 0; g < GP; ++g) {
                            const float2 *zg = Z + g * ZN;
                            const float2 A = zg[r * P + cx], B = zg[rm * P + cxm];
                            eh[j][2 * g] = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));      // (A + conj B) / 2
                            eh[j][2 * g + 1] = make_float2(0.5f * (A.y + B.y), 0.5f * (B.x - A.x));  // (A - conj B) / 2i
                        }
                    }
#pragma unroll
                    for (int j = 0; j < RA; ++j) {
                        const int row = row0 + j * RP;
                        if (row >= L) continue;
                        const bool lowrow = 2 * row <= L;
                        const int yr = lowrow ? row : L - row;
                        float2 run = av[j];
#pragma unroll
                        for (int e = 0; e < EG; ++e) {
                            if (e < ne) {
                                const float2 Gv = cmulc(eh[j][e], kv[j][e]);
                                run = cadd(run, Gv);
#pragma unroll
                                for (int k = 0; k < MS; ++k) {
                                    if (k < M) {
                                        const float2 *pgy = prof + prof_at(e, k, phy, 2, M, f, H);
                                        float2 gy = pgy[yr], gyd = pgy[H + yr];
                                        if (!lowrow) {
                                            gy.y = -gy.y;
                                            gyd.y = -gyd.y;
                                        }
                                        T1[e][k] = cadd(T1[e][k], cmulc(Gv, gy));
                                        T2[e][k] = cadd(T2[e][k], cmulc(Gv, gyd));
                                    }
                                }
                            }
                        }
                        st_hint(acc + ph * LHP + row * HP + tx, run, last ? pol_first : pol_last);
                    }
                }
#pragma unroll
                for (int e = 0; e < EG; ++e)
#pragma unroll
                    for (int k = 0; k < MS; ++k) {
                        if (k < M && e < ne) {
                            const float2 *pgx = prof + prof_at(e, k, phx, 0, M, f, H);
                            const float2 gx = pgx[tx], gxd = pgx[H + tx];
                            pa[e][k] += wgt * (T1[e][k].x * gx.x + T1[e][k].y * gx.y);
                            px[e][k] += wgt * (T1[e][k].x * gxd.x + T1[e][k].y * gxd.y);
                            py[e][k] += wgt * (T2[e][k].x * gx.x + T2[e][k].y * gx.y);
                        }
                    }
            }
        }
        __syncthreads();  // every read of Z is done: its first values take the per-warp partials
        float2 *red = Z;  // [value][warp]
        {
            const int g = warp % GP;
#pragma unroll
            for (int e = 0; e < EG; ++e) {
                if (e < ne) {
                    const bool mine = e / 2 == g;
                    const FSum c = mine ? chi[e & 1] : fsum_zero(), s = mine ? se[e & 1] : fsum_zero();
                    if (lane == 0) {
                        red[(e * nv + 0) * nw + warp] = make_float2(c.hi, c.lo);
                        red[(e * nv + 1) * nw + warp] = make_float2(s.hi, s.lo);
                    }
#pragma unroll
                    for (int k = 0; k < MS; ++k) {
                        if (k < M) {
                            float a = pa[e][k], bx = px[e][k], by = py[e][k];
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                a += __shfl_down_sync(0xffffffffu, a, o);
                                bx += __shfl_down_sync(0xffffffffu, bx, o);
                                by += __shfl_down_sync(0xffffffffu, by, o);
                            }
                            if (lane == 0) {
                                red[(e * nv + 2 + 3 * k) * nw + warp] = make_float2(a, 0.f);
                                red[(e * nv + 3 + 3 * k) * nw + warp] = make_float2(bx, 0.f);
                                red[(e * nv + 4 + 3 * k) * nw + warp] = make_float2(by, 0.f);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // warp v sums value v's per-warp partials in a fixed shuffle tree
        for (int v = warp; v < ne * nv; v += nw) {
            const float2 part = lane < nw ? red[v * nw + lane] : make_float2(0.f, 0.f);
            const FSum tot = fsum_warp(FSum{part.x, part.y});
            if (lane == 0) {
                const double sum = fsum_value(tot);
                const int e = v / nv, q = v - e * nv;
                const int i = i0 + e;
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
                    else ps_du[2 * ps + which - 1] = apar[e * M + k] * sc;
                }
            }
        }
        __syncthreads();
    }
}

// shared memory of one variant fits the opt-in limit (about 227 KB less the static part)
template <int L, int GP, int MS>
__host__ __device__ constexpr bool pr_fits() {
    return (GP * Pr<L>::ZN + 2 * GP * MS * 2 * 4 * Pr<L>::H + L) * 8 <= 231000;
}
// the widest group of pairs compiled for one source: 4 or 2 pairs where they fit, else 1
template <int L>
__host__ __device__ constexpr int pr_gpmax() {
    return pr_fits<L, 4, 1>() ? 4 : pr_fits<L, 2, 1>() ? 2 : 1;
}

template <int L>
__device__ __forceinline__ void chunk_item_dispatch(const FieldDev &fd, const int4 item, const float *params,
                                                    const float2 *hhat, float2 *acc, double *chi_part,
                                                    double *se_part, float *ps_da, float *ps_du) {
    // variants (pairs per group, source bound): (pr_gpmax, 1) and (1, 1) for M <= 1, (1, 4) else
    constexpr int GM = pr_gpmax<L>();
    if (fd.M > 1) {
        if constexpr (pr_fits<L, 1, kFftMaxSources>())
            chunk_item_pair<L, 1, kFftMaxSources>(fd, item, params, hhat, acc, chi_part, se_part, ps_da, ps_du);
    } else if (GM > 1 && fd.fft_G == GM) {
        chunk_item_pair<L, GM, 1>(fd, item, params, hhat, acc, chi_part, se_part, ps_da, ps_du);
    } else {
        chunk_item_pair<L, 1, 1>(fd, item, params, hhat, acc, chi_part, se_part, ps_da, ps_du);
    }
}

__global__ void __launch_bounds__(kFftThreads, 1)
fft_chunk_pair_kernel(const FieldDev *__restrict__ fields, const int4 *__restrict__ items, int n_items,
                      int *__restrict__ counter, const float *__restrict__ params, const float2 *__restrict__ hhat_all,
                      float2 *__restrict__ acc_all, double *__restrict__ chi_part, double *__restrict__ se_part,
                      float *__restrict__ ps_da, float *__restrict__ ps_du) {
    for (;;) {
        if (threadIdx.x == 0) pr_sh.item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = pr_sh.item;
        if (it >= n_items) break;
        const int4 item = items[it];
        const FieldDev &fd = fields[item.x];
        switch (fd.fft_L) {
#define SR_PR_CASE(LL)                                                                                      \
    case LL:                                                                                                \
        chunk_item_dispatch<LL>(fd, item, params, hhat_all, acc_all, chi_part, se_part, ps_da, ps_du);      \
        break;
            SR_PR_SIZES(SR_PR_CASE)
#undef SR_PR_CASE
            default:
                break;  // not reached: the host only builds items for sizes in the list
        }
        __syncthreads();
    }
}

template <int L>
constexpr int pair_zn() {
    return Pr<L>::ZN;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
bool fft_pair_size(int L) {
    switch (L) {
#define SR_PR_OK(LL) case LL:
        SR_PR_SIZES(SR_PR_OK)
#undef SR_PR_OK
        return true;
        default:
            return false;
    }
}

int fft_pair_next(int need) {
    static const int sizes[] = {
#define SR_PR_LIST(LL) LL,
        SR_PR_SIZES(SR_PR_LIST)
#undef SR_PR_LIST
    };
    for (int L : sizes)
        if (L >= need) return L;
    return 0;
}

int fft_pair_zn(int L) {
    switch (L) {
#define SR_PR_ZN(LL) \
    case LL:         \
        return pair_zn<LL>();
        SR_PR_SIZES(SR_PR_ZN)
#undef SR_PR_ZN
        default:
            return 0;
    }
}

// GP pair arrays, the window-profile tables of 2 GP epochs and the twiddles.
int fft_pair_smem_bytes(int L, int M, int f, int GP) {
    const int H = L / 2 + 1;
    return (GP * fft_pair_zn(L) + 2 * GP * M * f * 4 * H + L) * (int)sizeof(float2);
}

// The per-field and per-PSF kernels: one pair array and the twiddles.
int fft_pair_field_smem(int L) { return (fft_pair_zn(L) + L) * (int)sizeof(float2); }

// The widest group of epoch pairs the chunk kernel is compiled for at size L (one source).
int fft_pair_gpmax(int L) {
    switch (L) {
#define SR_PR_GM(LL) \
    case LL:         \
        return pr_gpmax<LL>();
        SR_PR_SIZES(SR_PR_GM)
#undef SR_PR_GM
        default:
            return 1;
    }
}

// Whether the chunk kernel has a compiled variant for (L, M, GP): one pair per group, or (for at
// most one source) the widest group of the size; more than one source needs the four-source
// variant to fit.
bool fft_pair_variant(int L, int M, int GP) {
    if (!fft_pair_size(L) || M > kFftMaxSources) return false;
    if (M > 1) {
        const int H = L / 2 + 1;
        return GP == 1 && (fft_pair_zn(L) + 2 * kFftMaxSources * 2 * 4 * H + L) * 8 <= 231000;
    }
    return GP == 1 || GP == fft_pair_gpmax(L);
}

template <typename K>
static sr_status open_smem(K kernel, int optin, int *limit) {
    cudaFuncAttributes a;
    SR_CUDA(cudaFuncGetAttributes(&a, kernel));
    const int dyn = optin - (int)a.sharedSizeBytes;
    SR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    *limit = std::min(*limit, dyn);
    return SR_OK;
}

// Fills the DFT twiddle tables and opens the largest dynamic shared memory each kernel can take;
// *chunk_limit and *field_limit are what the chunk kernel and the per-field kernels may use.
sr_status configure_fft_pair(int optin, int *chunk_limit, int *field_limit) {
    SR_CUDA(pr_fill_dtw());
    *chunk_limit = optin;
    sr_status s;
    if ((s = open_smem(fft_chunk_pair_kernel, optin, chunk_limit)) != SR_OK) return s;
    return configure_fft_pair_field(optin, field_limit);
}





sr_status occupancy_fft_pair(int smem, int *blocks) {
    SR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fft_chunk_pair_kernel, kFftThreads, smem));
    return SR_OK;
}

void launch_fft_chunks_pair(const FieldDev *fields, const int4 *items, int n_items, int *counter, const float *params,
                            const float2 *hhat, float2 *acc, double *chi_part, double *se_part, float *ps_da,
                            float *ps_du, int grid, int smem, cudaStream_t st) {
    fft_chunk_pair_kernel<<<grid, kFftThreads, smem, st>>>(fields, items, n_items, counter, params, hhat, acc,
                                                           chi_part, se_part, ps_da, ps_du);
}

}  // namespace sr
