// L-BFGS-B (the paper's second optimiser, sec. 2.4), from Byrd, Lu, Nocedal & Zhu (1995), "A
// limited memory algorithm for bound constrained optimization", SIAM J. Sci. Comput. 16(5).
//
// The limited-memory matrix is kept in compact form, B = theta I - W M W^T with W = [Y, theta S]
// (n x 2k, the k stored pairs) and M the inverse of [[-D, L^T], [L, theta S^T S]] (2k x 2k).
// The device holds the n-vectors: the parameters, the gradient, the trial point and gradient,
// the search direction and the pairs S, Y (column j at offset j n of a set of m + 1 columns).
// Everything n-long runs in the kernels below; the small algebra (2k x 2k) runs on the host in
// FP64.  The bounds of the problems this library optimises are lower bounds on a few contiguous
// ranges of the parameter vector (the amplitudes of each field; for a PSF fit also the Moffat alpha
// and beta), so the breakpoints of the generalised Cauchy point are those of the bounded set: a
// gather kernel packs its x, g and rows of W, the host sorts its breakpoints and walks them in
// order, and corrects the all-variable reductions for the variables it fixes at their bounds.
//
// Per iteration:
//   lbfgs_coldots_kernel   W^T g and g^T g (the Cauchy path's p = W^T d and f' = -d^T d)
//   (host)                 breakpoints of the bounded range, the Cauchy point x^c, c = W^T(x^c-x),
//                          the subspace system (W_Z^T W_Z = W^T W minus the fixed rows, W_Z^T r^c
//                          from W^T g, the fixed rows and x^c), v, the backtrack step alpha*
//   lbfgs_dir_kernel       d = x^c - x + alpha* du on the free variables, du = -r^c/theta -
//                          W v / theta^2, r^c = g + theta (x^c - x) - W M c
//   line search            lbfgs_axpy_kernel (x + a d), the library's loss and gradient, g^T d
//                          (strong Wolfe bracketing and zoom by bisection, Nocedal & Wright
//                          Algorithms 3.5-3.6, c1 = 1e-3, c2 = 0.9, steps in (0, 1])
//   lbfgs_pair_kernel      s = x_new - x, y = g_new - g into the ring, and their inner products
//                          with every stored column (the new rows of S^T S, S^T Y, Y^T S, Y^T Y)
// Reductions are FP64 per block in a fixed order, then summed on the host in block order.
#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>
#include <vector>

#include "lbfgsb.cuh"

namespace sr {
namespace {

constexpr int kLbThreads = 256;
constexpr int kLbMaxDots = 4 * kLbfgsMaxMemory + 3;

// out[b * J + j] = sum over block b's elements of A_j[i] * v[i] (A_j = cols[j])
struct ColPtrs {
    const float *p[kLbMaxDots];
    const float *q[kLbMaxDots];
};

__global__ void __launch_bounds__(kLbThreads) lbfgs_coldots_kernel(ColPtrs cp, int J, long long n,
                                                                   double *__restrict__ part) {
    __shared__ double red[kLbThreads / 32][kLbMaxDots];
    double acc[kLbMaxDots];
#pragma unroll
    for (int j = 0; j < kLbMaxDots; ++j) acc[j] = 0.0;
    for (long long i = blockIdx.x * (long long)kLbThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kLbThreads)
#pragma unroll
        for (int j = 0; j < kLbMaxDots; ++j)
            if (j < J) acc[j] += (double)cp.p[j][i] * (double)cp.q[j][i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kLbMaxDots; ++j) {
        if (j >= J) break;
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += kLbThreads) {
        double v = 0.0;
        for (int w = 0; w < kLbThreads / 32; ++w) v += red[w][j];
        part[(long long)blockIdx.x * J + j] = v;
    }
}

__global__ void lbfgs_axpy_kernel(const float *__restrict__ x, const float *__restrict__ d, float a, long long n,
                                  float *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = fmaf(a, d[i], x[i]);
}

struct DirArgs {
    int k;              // stored pairs
    int slot[kLbfgsMaxMemory];  // ring column of pair j (oldest first)
    double theta, told, alpha;
    double u[2 * kLbfgsMaxMemory];  // M c
    double v[2 * kLbfgsMaxMemory];  // the subspace solution
};

// d_i = x^c_i - x_i + alpha* du_i (free) or x^c_i - x_i (fixed); outside the bounded range
// x^c_i = x_i - told g_i and every variable is free
__global__ void __launch_bounds__(kLbThreads) lbfgs_dir_kernel(DirArgs a, const float *__restrict__ x,
                                                               const float *__restrict__ g, const float *__restrict__ S,
                                                               const float *__restrict__ Y, long long n,
                                                               const int *__restrict__ ridx,
                                                               const float *__restrict__ xcR,
                                                               const unsigned char *__restrict__ fixR,
                                                               float *__restrict__ d) {
    for (long long i = blockIdx.x * (long long)kLbThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kLbThreads) {
        const int r = ridx[i];  // slot in the bounded set, -1 for an unbounded variable
        const double xi = x[i], gi = g[i];
        const double xci = r >= 0 ? (double)xcR[r] : xi - a.told * gi;
        if (r >= 0 && fixR[r]) {
            d[i] = (float)(xci - xi);
            continue;
        }
        double wu = 0.0, wv = 0.0;
        for (int j = 0; j < a.k; ++j) {
            const double yj = Y[(long long)a.slot[j] * n + i], sj = a.theta * (double)S[(long long)a.slot[j] * n + i];
            wu += yj * a.u[j] + sj * a.u[a.k + j];
            wv += yj * a.v[j] + sj * a.v[a.k + j];
        }
        const double rc = gi + a.theta * (xci - xi) - wu;
        const double du = -rc / a.theta - wv / (a.theta * a.theta);
        d[i] = (float)(xci - xi + a.alpha * du);
    }
}

// the bounded set packed: x, g and the k stored columns of Y then of S at its variables
__global__ void lbfgs_gather_kernel(const long long *__restrict__ rsrc, long long nR, const float *__restrict__ x,
                                    const float *__restrict__ g, const float *__restrict__ S,
                                    const float *__restrict__ Y, long long n, DirArgs a, float *__restrict__ ox,
                                    float *__restrict__ og, float *__restrict__ oW) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nR; j += (long long)gridDim.x * blockDim.x) {
        const long long i = rsrc[j];
        ox[j] = x[i];
        og[j] = g[i];
        for (int c = 0; c < a.k; ++c) {
            oW[(long long)c * nR + j] = Y[(long long)a.slot[c] * n + i];
            oW[(long long)(a.k + c) * nR + j] = S[(long long)a.slot[c] * n + i];
        }
    }
}

// bounded variables clipped into their bounds
__global__ void lbfgs_clip_kernel(const long long *__restrict__ rsrc, long long nR, const float *__restrict__ loR,
                                  float *__restrict__ x) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nR; j += (long long)gridDim.x * blockDim.x)
        x[rsrc[j]] = fmaxf(x[rsrc[j]], loR[j]);
}

// s = xn - x and y = gn - g into ring column `col`
__global__ void lbfgs_pair_kernel(const float *__restrict__ x, const float *__restrict__ xn, const float *__restrict__ g,
                                  const float *__restrict__ gn, long long n, float *__restrict__ s,
                                  float *__restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        s[i] = xn[i] - x[i];
        y[i] = gn[i] - g[i];
    }
}

__global__ void __launch_bounds__(kLbThreads) lbfgs_pgnorm_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ g, long long n,
                                                                  const int *__restrict__ ridx,
                                                                  const float *__restrict__ loR,
                                                                  float *__restrict__ part) {
    __shared__ float red[kLbThreads];
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)kLbThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kLbThreads) {
        float t = x[i] - g[i];
        if (ridx[i] >= 0) t = fmaxf(t, loR[ridx[i]]);
        m = fmaxf(m, fabsf(t - x[i]));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = kLbThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- host -------------------------------------------------------------------------------------

// Solve A x = b (dense, partial pivoting) in place; false if singular.
bool solve_dense(std::vector<double> A, std::vector<double> &b, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * b[j];
        b[c] = s / A[c * n + c];
    }
    return true;
}

bool invert_dense(const std::vector<double> &A, std::vector<double> &inv, int n) {
    inv.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        std::vector<double> e(n, 0.0);
        e[c] = 1.0;
        if (!solve_dense(A, e, n)) return false;
        for (int r = 0; r < n; ++r) inv[(size_t)r * n + c] = e[r];
    }
    return true;
}

struct Dev {
    std::vector<void *> p;
    ~Dev() {
        for (void *q : p) cudaFree(q);
    }
    template <class T> cudaError_t alloc(T **q, size_t count) {
        *q = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(q), std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) p.push_back(*q);
        return e;
    }
};

}  // namespace

sr_status lbfgsb_run(const LbfgsbProblem &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist, sr_lbfgsb_info *info,
                     cudaStream_t st) {
    const long long n = P.n, nR = (long long)P.lo.size();
    const int m = cfg.m;
    int sms = 0, dev = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nblk = (int)std::max(1LL, std::min<long long>((n + kLbThreads - 1) / kLbThreads, 2LL * sms));
    Dev D;
    float *g, *xt, *gt, *d, *S, *Y, *xcR, *loR, *pgpart, *gx, *gg_, *gW;
    unsigned char *fixR;
    double *part;
    int *ridx;
    long long *rsrc;
    cudaError_t e = D.alloc(&g, n);
    if (!e) e = D.alloc(&xt, n);
    if (!e) e = D.alloc(&gt, n);
    if (!e) e = D.alloc(&d, n);
    if (!e) e = D.alloc(&S, (size_t)n * (m + 1));  // m pairs and a column for the candidate pair
    if (!e) e = D.alloc(&Y, (size_t)n * (m + 1));
    if (!e) e = D.alloc(&xcR, nR);
    if (!e) e = D.alloc(&loR, nR);
    if (!e) e = D.alloc(&fixR, nR);
    if (!e) e = D.alloc(&ridx, n);
    if (!e) e = D.alloc(&rsrc, nR);
    if (!e) e = D.alloc(&gx, nR);
    if (!e) e = D.alloc(&gg_, nR);
    if (!e) e = D.alloc(&gW, (size_t)2 * m * nR);
    if (!e) e = D.alloc(&pgpart, nblk);
    if (!e) e = D.alloc(&part, (size_t)nblk * kLbMaxDots);
    if (e) {
        cudaGetLastError();
        set_error("sr_lbfgsb: device allocation failed: %s", cudaGetErrorString(e));
        return SR_ERR_OOM;
    }
    std::vector<float> hx(nR), hg(nR), hlo(P.lo.begin(), P.lo.end());
    // the bounded set: slot of each variable (-1 outside), variable of each slot
    {
        std::vector<int> hr((size_t)n, -1);
        std::vector<long long> hs;
        hs.reserve((size_t)nR);
        for (const auto &rg : P.ranges)
            for (long long i = rg.first; i < rg.second; ++i) {
                hr[(size_t)i] = (int)hs.size();
                hs.push_back(i);
            }
        if ((long long)hs.size() != nR) {
            set_error("sr_lbfgsb: %lld bounds for %zu bounded variables", nR, hs.size());
            return SR_ERR_ARG;
        }
        SR_CUDA(cudaMemcpyAsync(ridx, hr.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaMemcpyAsync(rsrc, hs.data(), sizeof(long long) * nR, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaMemcpyAsync(loR, hlo.data(), sizeof(float) * nR, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    const int gR = (int)std::max(1LL, std::min<long long>((nR + 255) / 256, 8LL * sms));
    if (nR > 0) lbfgs_clip_kernel<<<gR, 256, 0, st>>>(rsrc, nR, loR, x);

    auto dots = [&](const std::vector<std::pair<const float *, const float *>> &pr, std::vector<double> &out) -> sr_status {
        ColPtrs cp{};
        const int J = (int)pr.size();
        for (int j = 0; j < J; ++j) {
            cp.p[j] = pr[j].first;
            cp.q[j] = pr[j].second;
        }
        lbfgs_coldots_kernel<<<nblk, kLbThreads, 0, st>>>(cp, J, n, part);
        std::vector<double> hp((size_t)nblk * J);
        SR_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        out.assign(J, 0.0);
        for (int b = 0; b < nblk; ++b)
            for (int j = 0; j < J; ++j) out[j] += hp[(size_t)b * J + j];
        return SR_OK;
    };
    const int gb = (int)std::min<long long>((n + 255) / 256, 8LL * sms);
    double f = 0.0, ft = 0.0;
    sr_status rs;
    if ((rs = P.eval(x, g, &f)) != SR_OK) return rs;
    int evals = 1, it = 0, status = SR_LBFGSB_MAX_ITER;
    if (f_hist) f_hist[0] = f;
    // memory: ring slots oldest first; inner products among stored columns
    std::vector<int> slots;
    std::vector<std::vector<double>> SS, SY, YY;  // SY[i][j] = s_i . y_j
    double theta = 1.0, pg = 0.0;
    auto pgnorm = [&](double *out) -> sr_status {
        lbfgs_pgnorm_kernel<<<nblk, kLbThreads, 0, st>>>(x, g, n, ridx, loR, pgpart);
        std::vector<float> hp(nblk);
        SR_CUDA(cudaMemcpyAsync(hp.data(), pgpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        *out = *std::max_element(hp.begin(), hp.end());
        return SR_OK;
    };
    while (it < cfg.max_iter) {
        if ((rs = pgnorm(&pg)) != SR_OK) return rs;
        if (pg <= cfg.pgtol) {
            status = SR_LBFGSB_PGTOL;
            break;
        }
        const int k = (int)slots.size(), k2 = 2 * k;
        // M = inverse of [[-D, L^T], [L, theta S^T S]]
        std::vector<double> Minv;
        if (k > 0) {
            std::vector<double> K((size_t)k2 * k2, 0.0);
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    if (i == j) K[(size_t)i * k2 + j] = -SY[i][i];
                    if (i > j) {
                        K[(size_t)(k + i) * k2 + j] = SY[i][j];  // L
                        K[(size_t)j * k2 + (k + i)] = SY[i][j];  // L^T
                    }
                    K[(size_t)(k + i) * k2 + (k + j)] = theta * SS[i][j];
                }
            if (!invert_dense(K, Minv, k2)) {
                status = SR_LBFGSB_LINE_SEARCH;
                break;
            }
        }
        auto Mv = [&](const std::vector<double> &a) {
            std::vector<double> o(k2, 0.0);
            for (int i = 0; i < k2; ++i)
                for (int j = 0; j < k2; ++j) o[i] += Minv[(size_t)i * k2 + j] * a[j];
            return o;
        };
        auto dotv = [](const std::vector<double> &a, const std::vector<double> &b) {
            double s = 0.0;
            for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
            return s;
        };
        // W^T g and g^T g over every variable
        std::vector<std::pair<const float *, const float *>> pr;
        for (int j = 0; j < k; ++j) pr.push_back({Y + (long long)slots[j] * n, g});
        for (int j = 0; j < k; ++j) pr.push_back({S + (long long)slots[j] * n, g});
        pr.push_back({g, g});
        std::vector<double> dv;
        if ((rs = dots(pr, dv)) != SR_OK) return rs;
        std::vector<double> Wg(k2);
        for (int j = 0; j < k; ++j) {
            Wg[j] = dv[j];
            Wg[k + j] = theta * dv[k + j];
        }
        const double gg = dv[k2];
        // the bounded set on the host: x, g and the rows of W
        std::vector<float> hW((size_t)k2 * nR);
        if (nR > 0) {
            DirArgs ga{};
            ga.k = k;
            for (int j = 0; j < k; ++j) ga.slot[j] = slots[j];
            lbfgs_gather_kernel<<<gR, 256, 0, st>>>(rsrc, nR, x, g, S, Y, n, ga, gx, gg_, gW);
            SR_CUDA(cudaMemcpyAsync(hx.data(), gx, sizeof(float) * nR, cudaMemcpyDeviceToHost, st));
            SR_CUDA(cudaMemcpyAsync(hg.data(), gg_, sizeof(float) * nR, cudaMemcpyDeviceToHost, st));
            if (k2) SR_CUDA(cudaMemcpyAsync(hW.data(), gW, sizeof(float) * k2 * nR, cudaMemcpyDeviceToHost, st));
            SR_CUDA(cudaStreamSynchronize(st));
        }
        auto wrow = [&](long long i, std::vector<double> &w) {
            w.resize(k2);
            for (int j = 0; j < k; ++j) {
                w[j] = hW[(size_t)j * nR + i];
                w[k + j] = theta * (double)hW[(size_t)(k + j) * nR + i];
            }
        };
        // generalised Cauchy point: breakpoints of the bounded range
        std::vector<double> t(nR), dR(nR);
        std::vector<unsigned char> fix(nR, 0);
        std::vector<double> p(k2), c(k2, 0.0), w;
        for (int j = 0; j < k2; ++j) p[j] = -Wg[j];
        double fp = -gg;
        for (long long i = 0; i < nR; ++i) {
            const double gi = hg[i], xi = hx[i];
            t[i] = gi > 0 ? (xi - hlo[i]) / gi : INFINITY;
            dR[i] = -gi;
            if (t[i] == 0.0) {  // at the bound and pushed out: fixed, no motion
                fix[i] = 1;
                dR[i] = 0.0;
                fp += gi * gi;
                if (k) {
                    wrow(i, w);
                    for (int j = 0; j < k2; ++j) p[j] += gi * w[j];
                }
            }
        }
        double fpp = -theta * fp - (k ? dotv(p, Mv(p)) : 0.0);
        const double fpp0 = -theta * fp;
        double dtm = fpp > 0 ? -fp / fpp : 0.0, told = 0.0;
        std::vector<long long> order;
        for (long long i = 0; i < nR; ++i)
            if (std::isfinite(t[i]) && t[i] > 0) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return t[a] < t[b]; });
        std::vector<double> xcR_h(hx.begin(), hx.end());
        for (long long b : order) {
            const double tj = t[b], dt = tj - told;
            if (dtm < dt) break;
            const double xcb = hlo[b];  // lower bounds only
            const double zb = xcb - hx[b], gb_ = hg[b];
            if (k)
                for (int j = 0; j < k2; ++j) c[j] += dt * p[j];
            fp += dt * fpp + gb_ * gb_ + theta * gb_ * zb;
            fpp -= theta * gb_ * gb_;
            if (k) {
                wrow(b, w);
                const std::vector<double> Mc = Mv(c), Mp = Mv(p), Mw = Mv(w);
                fp -= gb_ * dotv(w, Mc);
                fpp -= 2.0 * gb_ * dotv(w, Mp) + gb_ * gb_ * dotv(w, Mw);
                for (int j = 0; j < k2; ++j) p[j] += gb_ * w[j];
            }
            fpp = std::max(2.220446049250313e-16 * fpp0, fpp);
            dR[b] = 0.0;
            fix[b] = 1;
            xcR_h[b] = xcb;
            dtm = fpp > 0 ? -fp / fpp : 0.0;
            told = tj;
        }
        dtm = std::max(dtm, 0.0);
        told += dtm;
        for (long long i = 0; i < nR; ++i)
            if (!fix[i]) xcR_h[i] = hx[i] + told * dR[i];
        if (k)
            for (int j = 0; j < k2; ++j) c[j] += dtm * p[j];
        // subspace minimisation over the free variables
        DirArgs da{};
        da.k = k;
        for (int j = 0; j < k; ++j) da.slot[j] = slots[j];
        da.theta = theta;
        da.told = told;
        std::vector<double> u(k2, 0.0), v(k2, 0.0);
        double alpha = 1.0;
        if (k) {
            u = Mv(c);
            // W^T W over every variable from the stored inner products
            std::vector<double> WW((size_t)k2 * k2);
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    WW[(size_t)i * k2 + j] = YY[i][j];
                    WW[(size_t)i * k2 + k + j] = theta * SY[j][i];
                    WW[(size_t)(k + i) * k2 + j] = theta * SY[i][j];
                    WW[(size_t)(k + i) * k2 + k + j] = theta * theta * SS[i][j];
                }
            // W^T (x^c - x): -told W^T g outside the range; exact inside it
            std::vector<double> Wdx(k2), WWu(k2, 0.0);
            for (int j = 0; j < k2; ++j) Wdx[j] = -told * Wg[j];
            for (long long i = 0; i < nR; ++i) {
                wrow(i, w);
                const double corr = (xcR_h[i] - hx[i]) + told * hg[i];
                for (int j = 0; j < k2; ++j) Wdx[j] += w[j] * corr;
            }
            for (int i = 0; i < k2; ++i)
                for (int j = 0; j < k2; ++j) WWu[i] += WW[(size_t)i * k2 + j] * u[j];
            // W_Z^T r^c and W_Z^T W_Z: every variable minus the fixed rows
            std::vector<double> Wr(k2), WzWz = WW;
            for (int j = 0; j < k2; ++j) Wr[j] = Wg[j] + theta * Wdx[j] - WWu[j];
            for (long long i = 0; i < nR; ++i) {
                if (!fix[i]) continue;
                wrow(i, w);
                const double rc = hg[i] + theta * (xcR_h[i] - hx[i]) - dotv(w, u);
                for (int a = 0; a < k2; ++a) {
                    Wr[a] -= w[a] * rc;
                    for (int b2 = 0; b2 < k2; ++b2) WzWz[(size_t)a * k2 + b2] -= w[a] * w[b2];
                }
            }
            v = Mv(Wr);
            std::vector<double> Nm((size_t)k2 * k2);
            for (int i = 0; i < k2; ++i)
                for (int j = 0; j < k2; ++j) {
                    double s = 0.0;
                    for (int l = 0; l < k2; ++l) s += Minv[(size_t)i * k2 + l] * WzWz[(size_t)l * k2 + j];
                    Nm[(size_t)i * k2 + j] = (i == j ? 1.0 : 0.0) - s / theta;
                }
            if (!solve_dense(Nm, v, k2)) {
                status = SR_LBFGSB_LINE_SEARCH;
                break;
            }
        }
        // backtrack into the box over the free bounded variables
        for (long long i = 0; i < nR; ++i) {
            if (fix[i]) continue;
            double wu = 0.0, wv = 0.0;
            if (k) {
                wrow(i, w);
                wu = dotv(w, u);
                wv = dotv(w, v);
            }
            const double rc = hg[i] + theta * (xcR_h[i] - hx[i]) - wu;
            const double du = -rc / theta - wv / (theta * theta);
            if (du < 0) alpha = std::min(alpha, (hlo[i] - xcR_h[i]) / du);
        }
        alpha = std::max(alpha, 0.0);
        for (int j = 0; j < k2; ++j) {
            da.u[j] = u[j];
            da.v[j] = v[j];
        }
        da.alpha = alpha;
        std::vector<float> xcR_f(nR);
        for (long long i = 0; i < nR; ++i) xcR_f[i] = (float)xcR_h[i];
        SR_CUDA(cudaMemcpyAsync(xcR, xcR_f.data(), sizeof(float) * nR, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaMemcpyAsync(fixR, fix.data(), nR, cudaMemcpyHostToDevice, st));
        lbfgs_dir_kernel<<<nblk, kLbThreads, 0, st>>>(da, x, g, S, Y, n, ridx, xcR, fixR, d);
        // line search along d
        std::vector<double> dd;
        if ((rs = dots({{d, d}, {g, d}}, dd)) != SR_OK) return rs;
        const double dn = std::sqrt(dd[0]), dphi0 = dd[1];
        if (dn == 0.0) {
            status = SR_LBFGSB_PGTOL;
            break;
        }
        if (!(dphi0 < 0.0)) {
            status = SR_LBFGSB_LINE_SEARCH;
            break;
        }
        const double c1 = 1e-3, c2 = 0.9;
        int ls = 0;
        auto phi = [&](double a, double *fa, double *dpa) -> sr_status {
            lbfgs_axpy_kernel<<<gb, 256, 0, st>>>(x, d, (float)a, n, xt);
            sr_status s2 = P.eval(xt, gt, fa);
            if (s2 != SR_OK) return s2;
            ++ls;
            std::vector<double> o;
            if ((s2 = dots({{gt, d}}, o)) != SR_OK) return s2;
            *dpa = o[0];
            return SR_OK;
        };
        bool found = false;
        double a_acc = 0.0;
        // the accepted trial must be the last one evaluated (xt, gt hold it); zoom re-evaluates
        auto zoom = [&](double alo, double flo, double ahi) -> sr_status {
            while (ls < cfg.max_ls) {
                const double a = 0.5 * (alo + ahi);
                double fa, dpa;
                sr_status s2 = phi(a, &fa, &dpa);
                if (s2 != SR_OK) return s2;
                if (fa > f + c1 * a * dphi0 || fa >= flo) {
                    ahi = a;
                } else {
                    if (std::fabs(dpa) <= -c2 * dphi0) {
                        found = true;
                        a_acc = a;
                        ft = fa;
                        return SR_OK;
                    }
                    if (dpa * (ahi - alo) >= 0) ahi = alo;
                    alo = a;
                    flo = fa;
                }
            }
            return SR_OK;
        };
        double a_prev = 0.0, f_prev = f, a = it == 0 ? std::min(1.0, 1.0 / dn) : 1.0;
        while (ls < cfg.max_ls && !found) {
            double fa, dpa;
            if ((rs = phi(a, &fa, &dpa)) != SR_OK) return rs;
            if (fa > f + c1 * a * dphi0 || (a_prev > 0 && fa >= f_prev)) {
                if ((rs = zoom(a_prev, f_prev, a)) != SR_OK) return rs;
                break;
            }
            if (std::fabs(dpa) <= -c2 * dphi0) {
                found = true;
                a_acc = a;
                ft = fa;
                break;
            }
            if (dpa >= 0) {
                if ((rs = zoom(a, fa, a_prev)) != SR_OK) return rs;
                break;
            }
            if (a >= 1.0) {  // the whole step is feasible and still descending
                found = true;
                a_acc = a;
                ft = fa;
                break;
            }
            a_prev = a;
            f_prev = fa;
            a = std::min(2.0 * a, 1.0);
        }
        evals += ls;
        if (!found) {
            status = SR_LBFGSB_LINE_SEARCH;
            break;
        }
        (void)a_acc;
        // the candidate pair, into a column no stored pair uses
        int col = 0;
        while (std::find(slots.begin(), slots.end(), col) != slots.end()) ++col;
        float *sc = S + (long long)col * n, *yc = Y + (long long)col * n;
        lbfgs_pair_kernel<<<gb, 256, 0, st>>>(x, xt, g, gt, n, sc, yc);
        std::vector<std::pair<const float *, const float *>> pp = {{sc, yc}, {yc, yc}, {sc, sc}};
        for (int j = 0; j < k; ++j) {
            const float *Sj = S + (long long)slots[j] * n, *Yj = Y + (long long)slots[j] * n;
            pp.push_back({sc, Sj});
            pp.push_back({sc, Yj});
            pp.push_back({Sj, yc});
            pp.push_back({yc, Yj});
        }
        std::vector<double> o;
        if ((rs = dots(pp, o)) != SR_OK) return rs;
        const double sy = o[0], yy = o[1], ss = o[2];
        if (sy > 2.220446049250313e-16 * yy) {
            int keep0 = 0;
            if (k == m) {  // drop the oldest
                keep0 = 1;
                slots.erase(slots.begin());
                SS.erase(SS.begin());
                SY.erase(SY.begin());
                YY.erase(YY.begin());
                for (auto &r : SS) r.erase(r.begin());
                for (auto &r : SY) r.erase(r.begin());
                for (auto &r : YY) r.erase(r.begin());
            }
            const int kk = (int)slots.size();
            for (int j = 0; j < kk; ++j) {
                const size_t b = 3 + 4 * (size_t)(j + keep0);
                SS[j].push_back(o[b]);      // s_j . s_new
                SY[j].push_back(o[b + 2]);  // s_j . y_new
                YY[j].push_back(o[b + 3]);  // y_j . y_new
            }
            std::vector<double> rS, rSY, rY;
            for (int j = 0; j < kk; ++j) {
                const size_t b = 3 + 4 * (size_t)(j + keep0);
                rS.push_back(o[b]);
                rSY.push_back(o[b + 1]);  // s_new . y_j
                rY.push_back(o[b + 3]);
            }
            rS.push_back(ss);
            rSY.push_back(sy);
            rY.push_back(yy);
            SS.push_back(rS);
            SY.push_back(rSY);
            YY.push_back(rY);
            slots.push_back(col);
            theta = yy / sy;
        }
        SR_CUDA(cudaMemcpyAsync(x, xt, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        std::swap(g, gt);
        const double fo = f;
        f = ft;
        ++it;
        if (f_hist) f_hist[it] = f;
        if ((fo - f) / std::max({std::fabs(fo), std::fabs(f), 1.0}) <= cfg.factr * 2.220446049250313e-16) {
            status = SR_LBFGSB_FACTR;
            break;
        }
    }
    if (status != SR_LBFGSB_PGTOL && (rs = pgnorm(&pg)) != SR_OK) return rs;
    SR_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = it;
        info->evaluations = evals;
        info->status = status;
        info->f = f;
        info->pg_norm = pg;
    }
    return SR_OK;
}

}  // namespace sr
