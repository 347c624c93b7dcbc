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
#include <thread>
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

// ---- per-field engine (independent runs over the fields of a batch) ---------------------------

// A chunk of one field's segment of the packed vector.
struct SegChunk {
    int field;
    long long beg, end;
};

constexpr int kLbVecs = 2 * (kLbfgsMaxMemory + 1) + 5;  // x, g, xt, gt, d, the S and Y columns

struct VecTable {
    const float *v[kLbVecs];
};

// part[c * J + q] = sum over chunk c of vecs[codes[f J + q].x] * vecs[codes[f J + q].y], f the
// chunk's field (FP64 in a fixed order: per thread, a warp tree, warps in order)
__global__ void __launch_bounds__(kLbThreads) lbf_segdots_kernel(const SegChunk *__restrict__ chunks, VecTable vt,
                                                                 const uchar2 *__restrict__ codes, int J,
                                                                 double *__restrict__ part) {
    __shared__ double red[kLbThreads / 32][kLbMaxDots];
    __shared__ const float *s_a[kLbMaxDots], *s_b[kLbMaxDots];
    const SegChunk ch = chunks[blockIdx.x];
    if (threadIdx.x < J) {
        const uchar2 c = codes[(long long)ch.field * J + threadIdx.x];
        s_a[threadIdx.x] = vt.v[c.x];
        s_b[threadIdx.x] = vt.v[c.y];
    }
    __syncthreads();
    double acc[kLbMaxDots];
#pragma unroll
    for (int j = 0; j < kLbMaxDots; ++j) acc[j] = 0.0;
    for (long long i = ch.beg + threadIdx.x; i < ch.end; i += kLbThreads)
#pragma unroll
        for (int j = 0; j < kLbMaxDots; ++j)
            if (j < J) acc[j] += (double)s_a[j][i] * (double)s_b[j][i];
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

// part[c] = max over chunk c of |P(x - g) - x| (P the projection onto the bounds)
__global__ void __launch_bounds__(kLbThreads) lbf_pgnorm_kernel(const SegChunk *__restrict__ chunks,
                                                                const float *__restrict__ x,
                                                                const float *__restrict__ g,
                                                                const int *__restrict__ ridx,
                                                                const float *__restrict__ loR,
                                                                float *__restrict__ part) {
    __shared__ float red[kLbThreads];
    const SegChunk ch = chunks[blockIdx.x];
    float m = 0.f;
    for (long long i = ch.beg + threadIdx.x; i < ch.end; i += kLbThreads) {
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

// xt = x + a_f d, a_f the step of the element's field
__global__ void lbf_axpy_kernel(const float *__restrict__ x, const float *__restrict__ d, const float *__restrict__ a,
                                const int *__restrict__ fid, long long n, float *__restrict__ xt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        xt[i] = fmaf(a[fid[i]], d[i], x[i]);
}

// the direction of each active field (inactive fields: d = 0); as lbfgs_dir_kernel with the
// arguments of the element's field
__global__ void __launch_bounds__(kLbThreads) lbf_dir_kernel(const DirArgs *__restrict__ args,
                                                             const unsigned char *__restrict__ active,
                                                             const int *__restrict__ fid, const float *__restrict__ x,
                                                             const float *__restrict__ g, const float *__restrict__ S,
                                                             const float *__restrict__ Y, long long n,
                                                             const int *__restrict__ ridx,
                                                             const float *__restrict__ xcR,
                                                             const unsigned char *__restrict__ fixR,
                                                             float *__restrict__ d) {
    for (long long i = blockIdx.x * (long long)kLbThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kLbThreads) {
        const int f = fid[i];
        if (!active[f]) {
            d[i] = 0.f;
            continue;
        }
        const DirArgs &a = args[f];
        const int r = ridx[i];
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

// the bounded set packed, with the rows of W of each variable's field (k_f columns of Y, then of S)
__global__ void lbf_gather_kernel(const long long *__restrict__ rsrc, const int *__restrict__ rfid, long long nR,
                                  const DirArgs *__restrict__ args, const float *__restrict__ x,
                                  const float *__restrict__ g, const float *__restrict__ S,
                                  const float *__restrict__ Y, long long n, float *__restrict__ ox,
                                  float *__restrict__ og, float *__restrict__ oW) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nR; j += (long long)gridDim.x * blockDim.x) {
        const long long i = rsrc[j];
        const DirArgs &a = args[rfid[j]];
        ox[j] = x[i];
        og[j] = g[i];
        for (int c = 0; c < a.k; ++c) {
            oW[(long long)c * nR + j] = Y[(long long)a.slot[c] * n + i];
            oW[(long long)(a.k + c) * nR + j] = S[(long long)a.slot[c] * n + i];
        }
    }
}

// the candidate pair of each field that took a step into its column col[f] (>= 0); then the step
// taken: x = xt, g = gt on those fields
__global__ void lbf_pair_kernel(const int *__restrict__ col, const int *__restrict__ fid, const float *__restrict__ x,
                                const float *__restrict__ xt, const float *__restrict__ g,
                                const float *__restrict__ gt, long long n, float *__restrict__ S,
                                float *__restrict__ Y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = col[fid[i]];
        if (c < 0) continue;
        S[(long long)c * n + i] = xt[i] - x[i];
        Y[(long long)c * n + i] = gt[i] - g[i];
    }
}

__global__ void lbf_accept_kernel(const int *__restrict__ col, const int *__restrict__ fid, const float *__restrict__ xt,
                                  const float *__restrict__ gt, long long n, float *__restrict__ x,
                                  float *__restrict__ g) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (col[fid[i]] < 0) continue;
        x[i] = xt[i];
        g[i] = gt[i];
    }
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

// The limited memory of one run: ring columns of the stored pairs (oldest first), their inner
// products and theta.
struct Memory {
    std::vector<int> slots;
    std::vector<std::vector<double>> SS, SY, YY;  // SY[i][j] = s_i . y_j
    double theta = 1.0;
};

// The bounded rows of one run on the host: x, g and the bounds at its nR bounded variables, and
// column c of W at row i in W[c * stride + i] (k columns of Y, then k of S).
struct Rows {
    long long nR = 0;
    const float *x = nullptr, *g = nullptr, *lo = nullptr, *W = nullptr;
    long long stride = 0;
};

// The host half of one iteration: the generalised Cauchy point over the bounded rows, the direct
// primal subspace minimisation and the backtrack into the box (Byrd et al. 1995, sec. 4-5).
// Wg = W^T g over every variable (2k values, theta already applied to the S half), gg = g^T g.
// Fills da (k, slots, theta, told, u = M c, v, alpha) and, per bounded row, xc and whether it is
// fixed.  Returns false when a 2k x 2k system is singular.
bool cauchy_subspace(const Memory &mem, const std::vector<double> &Wg, double gg, const Rows &R, DirArgs &da,
                     float *xcR_out, unsigned char *fix_out) {
    const int k = (int)mem.slots.size(), k2 = 2 * k;
    const double theta = mem.theta;
    const long long nR = R.nR;
    const auto &SS = mem.SS, &SY = mem.SY, &YY = mem.YY;
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
        if (!invert_dense(K, Minv, k2)) return false;
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
    auto wrow = [&](long long i, std::vector<double> &w) {
        w.resize(k2);
        for (int j = 0; j < k; ++j) {
            w[j] = R.W[(size_t)j * R.stride + i];
            w[k + j] = theta * (double)R.W[(size_t)(k + j) * R.stride + i];
        }
    };
    const float *hx = R.x, *hg = R.g, *hlo = R.lo;
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
    std::vector<double> xcR_h(hx, hx + nR);
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
    da = DirArgs{};
    da.k = k;
    for (int j = 0; j < k; ++j) da.slot[j] = mem.slots[j];
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
        if (!solve_dense(Nm, v, k2)) return false;
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
    for (long long i = 0; i < nR; ++i) {
        xcR_out[i] = (float)xcR_h[i];
        fix_out[i] = fix[i];
    }
    return true;
}

// The dots of a candidate pair (s, y) in column `col` against the stored pairs: s.y, y.y, s.s, then
// per stored pair j (oldest first) s.S_j, s.Y_j, S_j.y, y.Y_j.  push_pair keeps it when
// s.y > eps y.y (dropping the oldest pair at m pairs) and sets theta = y.y / s.y.
void push_pair(Memory &mem, int m, int col, const double *o) {
    const int k = (int)mem.slots.size();
    const double sy = o[0], yy = o[1], ss = o[2];
    if (!(sy > 2.220446049250313e-16 * yy)) return;
    auto &SS = mem.SS, &SY = mem.SY, &YY = mem.YY;
    int keep0 = 0;
    if (k == m) {  // drop the oldest
        keep0 = 1;
        mem.slots.erase(mem.slots.begin());
        SS.erase(SS.begin());
        SY.erase(SY.begin());
        YY.erase(YY.begin());
        for (auto &r : SS) r.erase(r.begin());
        for (auto &r : SY) r.erase(r.begin());
        for (auto &r : YY) r.erase(r.begin());
    }
    const int kk = (int)mem.slots.size();
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
    mem.slots.push_back(col);
    mem.theta = yy / sy;
}

// the first ring column (of m + 1) that no stored pair uses
int free_column(const Memory &mem) {
    int col = 0;
    while (std::find(mem.slots.begin(), mem.slots.end(), col) != mem.slots.end()) ++col;
    return col;
}

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
    Memory mem;
    double pg = 0.0;
    auto pgnorm = [&](double *out) -> sr_status {
        lbfgs_pgnorm_kernel<<<nblk, kLbThreads, 0, st>>>(x, g, n, ridx, loR, pgpart);
        std::vector<float> hp(nblk);
        SR_CUDA(cudaMemcpyAsync(hp.data(), pgpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        *out = *std::max_element(hp.begin(), hp.end());
        return SR_OK;
    };
    std::vector<float> xcR_f(nR);
    std::vector<unsigned char> fix(nR);
    while (it < cfg.max_iter) {
        if ((rs = pgnorm(&pg)) != SR_OK) return rs;
        if (pg <= cfg.pgtol) {
            status = SR_LBFGSB_PGTOL;
            break;
        }
        const int k = (int)mem.slots.size(), k2 = 2 * k;
        const std::vector<int> &slots = mem.slots;
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
            Wg[k + j] = mem.theta * dv[k + j];
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
        Rows R;
        R.nR = nR;
        R.x = hx.data();
        R.g = hg.data();
        R.lo = hlo.data();
        R.W = hW.data();
        R.stride = nR;
        DirArgs da{};
        if (!cauchy_subspace(mem, Wg, gg, R, da, xcR_f.data(), fix.data())) {
            status = SR_LBFGSB_LINE_SEARCH;
            break;
        }
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
                ft = fa;
                break;
            }
            if (dpa >= 0) {
                if ((rs = zoom(a, fa, a_prev)) != SR_OK) return rs;
                break;
            }
            if (a >= 1.0) {  // the whole step is feasible and still descending
                found = true;
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
        // the candidate pair, into a column no stored pair uses
        const int col = free_column(mem);
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
        push_pair(mem, m, col, o.data());
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

namespace {

// Line-search state of one field (the bracketing phase and the zoom of lbfgsb_run as a machine
// that takes one evaluation per round).
struct FieldSearch {
    bool searching = false, found = false;
    bool zoom = false;
    int ls = 0;
    double f0 = 0.0, dphi0 = 0.0;  // loss and directional derivative at the step's origin
    double a = 0.0, a_prev = 0.0, f_prev = 0.0, alo = 0.0, flo = 0.0, ahi = 0.0, ft = 0.0;
};

// The next state after the evaluation of trial a (loss fa, directional derivative dpa), with the
// tests of lbfgsb_run: c1 = 1e-3, c2 = 0.9, bisection in the zoom, doubling up to 1 in the bracket.
void search_update(FieldSearch &s, double fa, double dpa, int max_ls) {
    const double c1 = 1e-3, c2 = 0.9;
    ++s.ls;
    const double a = s.a;
    if (!s.zoom) {
        if (fa > s.f0 + c1 * a * s.dphi0 || (s.a_prev > 0 && fa >= s.f_prev)) {
            s.zoom = true;
            s.alo = s.a_prev;
            s.flo = s.f_prev;
            s.ahi = a;
        } else if (std::fabs(dpa) <= -c2 * s.dphi0) {
            s.found = true;
        } else if (dpa >= 0) {
            s.zoom = true;
            s.alo = a;
            s.flo = fa;
            s.ahi = s.a_prev;
        } else if (a >= 1.0) {
            s.found = true;
        } else {
            s.a_prev = a;
            s.f_prev = fa;
            s.a = std::min(2.0 * a, 1.0);
        }
    } else {
        if (fa > s.f0 + c1 * a * s.dphi0 || fa >= s.flo) {
            s.ahi = a;
        } else if (std::fabs(dpa) <= -c2 * s.dphi0) {
            s.found = true;
        } else {
            if (dpa * (s.ahi - s.alo) >= 0) s.ahi = s.alo;
            s.alo = a;
            s.flo = fa;
        }
    }
    if (s.found) {
        s.ft = fa;
        s.searching = false;
        return;
    }
    if (s.zoom) s.a = 0.5 * (s.alo + s.ahi);
    if (s.ls >= max_ls) s.searching = false;  // no strong-Wolfe step within max_ls evaluations
}

// Run fn(i) for i in [0, n) on up to `threads` host threads (static partition, in order within
// each thread); fn must not touch another index's data.
void parallel_for(int n, int threads, const std::function<void(int)> &fn) {
    threads = std::max(1, std::min(threads, n));
    if (threads == 1) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t]() {
            for (int i = t; i < n; i += threads) fn(i);
        });
    for (auto &th : pool) th.join();
}

}  // namespace

sr_status lbfgsb_fields_run(const LbfgsbFields &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist,
                            sr_lbfgsb_info *info, int *rounds_out, cudaStream_t st) {
    const long long n = P.n;
    const int nf = (int)P.off.size(), m = cfg.m;
    int sms = 0, dev = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // per-field segments and bounded rows; chunks of at most 16384 elements per field
    constexpr long long kChunk = 16384;
    std::vector<SegChunk> hch;
    std::vector<int> c0(nf + 1, 0);
    std::vector<long long> r0(nf + 1, 0);
    std::vector<int> hfid((size_t)n, -1), hr((size_t)n, -1), hrfid;
    std::vector<long long> hs;
    std::vector<float> hlo;
    for (int f = 0; f < nf; ++f) {
        c0[f] = (int)hch.size();
        for (long long b = P.off[f]; b < P.off[f] + P.len[f]; b += kChunk)
            hch.push_back({f, b, std::min(b + kChunk, P.off[f] + P.len[f])});
        for (long long i = P.off[f]; i < P.off[f] + P.len[f]; ++i) hfid[(size_t)i] = f;
        r0[f] = (long long)hs.size();
        for (const auto &rg : P.ranges[f])
            for (long long i = rg.first; i < rg.second; ++i) {
                hr[(size_t)i] = (int)hs.size();
                hs.push_back(i);
                hrfid.push_back(f);
            }
        hlo.insert(hlo.end(), P.lo[f].begin(), P.lo[f].end());
        if ((long long)hs.size() - r0[f] != (long long)P.lo[f].size()) {
            set_error("sr_batch_lbfgsb_fields: field %d has %zu bounds for %lld bounded variables", f, P.lo[f].size(),
                      (long long)hs.size() - r0[f]);
            return SR_ERR_ARG;
        }
    }
    c0[nf] = (int)hch.size();
    r0[nf] = (long long)hs.size();
    for (long long i = 0; i < n; ++i)
        if (hfid[(size_t)i] < 0) {
            set_error("sr_batch_lbfgsb_fields: parameter %lld belongs to no field", i);
            return SR_ERR_ARG;
        }
    const long long nR = (long long)hs.size();
    const int nch = (int)hch.size();
    Dev D;
    float *g, *xt, *gt, *d, *S, *Y, *xcR, *loR, *pgpart, *gx, *gg_, *gW, *astep;
    unsigned char *fixR, *act;
    double *part, *losses;
    int *ridx, *fid, *rfid, *colv;
    long long *rsrc;
    SegChunk *chunks;
    uchar2 *codes;
    DirArgs *dargs;
    cudaError_t e = D.alloc(&g, n);
    if (!e) e = D.alloc(&xt, n);
    if (!e) e = D.alloc(&gt, n);
    if (!e) e = D.alloc(&d, n);
    if (!e) e = D.alloc(&S, (size_t)n * (m + 1));
    if (!e) e = D.alloc(&Y, (size_t)n * (m + 1));
    if (!e) e = D.alloc(&xcR, nR);
    if (!e) e = D.alloc(&loR, nR);
    if (!e) e = D.alloc(&fixR, nR);
    if (!e) e = D.alloc(&ridx, n);
    if (!e) e = D.alloc(&fid, n);
    if (!e) e = D.alloc(&rsrc, nR);
    if (!e) e = D.alloc(&rfid, nR);
    if (!e) e = D.alloc(&gx, nR);
    if (!e) e = D.alloc(&gg_, nR);
    if (!e) e = D.alloc(&gW, (size_t)2 * m * nR);
    if (!e) e = D.alloc(&pgpart, nch);
    if (!e) e = D.alloc(&part, (size_t)nch * kLbMaxDots);
    if (!e) e = D.alloc(&losses, nf);
    if (!e) e = D.alloc(&astep, nf);
    if (!e) e = D.alloc(&act, nf);
    if (!e) e = D.alloc(&colv, nf);
    if (!e) e = D.alloc(&chunks, nch);
    if (!e) e = D.alloc(&codes, (size_t)nf * kLbMaxDots);
    if (!e) e = D.alloc(&dargs, nf);
    if (e) {
        cudaGetLastError();
        set_error("sr_batch_lbfgsb_fields: device allocation failed: %s", cudaGetErrorString(e));
        return SR_ERR_OOM;
    }
    SR_CUDA(cudaMemcpyAsync(ridx, hr.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(fid, hfid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(rsrc, hs.data(), sizeof(long long) * nR, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(rfid, hrfid.data(), sizeof(int) * nR, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(loR, hlo.data(), sizeof(float) * nR, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(chunks, hch.data(), sizeof(SegChunk) * nch, cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaStreamSynchronize(st));
    const int gR = (int)std::max(1LL, std::min<long long>((nR + 255) / 256, 8LL * sms));
    const int gb = (int)std::max(1LL, std::min<long long>((n + 255) / 256, 8LL * sms));
    if (nR > 0) lbfgs_clip_kernel<<<gR, 256, 0, st>>>(rsrc, nR, loR, x);

    // vector table: 0 x, 1 g, 2 xt, 3 gt, 4 d, 5 + c the S column c, 6 + m + c the Y column c
    VecTable vt{};
    vt.v[0] = x;
    vt.v[1] = g;
    vt.v[2] = xt;
    vt.v[3] = gt;
    vt.v[4] = d;
    for (int c = 0; c <= m; ++c) {
        vt.v[5 + c] = S + (long long)c * n;
        vt.v[6 + m + c] = Y + (long long)c * n;
    }
    const unsigned char VG = 1, VGT = 3, VD = 4;  // g, gt, d
    auto vS = [&](int c) { return (unsigned char)(5 + c); };
    auto vY = [&](int c) { return (unsigned char)(6 + m + c); };
    // per-field dot lists (J per field, shorter lists padded with g.g), summed per field in chunk order
    auto segdots = [&](const std::vector<std::vector<uchar2>> &lists, std::vector<std::vector<double>> &out) -> sr_status {
        int J = 1;
        for (const auto &l : lists) J = std::max(J, (int)l.size());
        std::vector<uchar2> hc((size_t)nf * J, make_uchar2(VG, VG));
        for (int f = 0; f < nf; ++f)
            for (size_t q = 0; q < lists[f].size(); ++q) hc[(size_t)f * J + q] = lists[f][q];
        SR_CUDA(cudaMemcpyAsync(codes, hc.data(), sizeof(uchar2) * hc.size(), cudaMemcpyHostToDevice, st));
        lbf_segdots_kernel<<<nch, kLbThreads, 0, st>>>(chunks, vt, codes, J, part);
        std::vector<double> hp((size_t)nch * J);
        SR_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        out.assign(nf, {});
        for (int f = 0; f < nf; ++f) {
            out[f].assign(lists[f].size(), 0.0);
            for (int c = c0[f]; c < c0[f + 1]; ++c)
                for (size_t q = 0; q < lists[f].size(); ++q) out[f][q] += hp[(size_t)c * J + q];
        }
        return SR_OK;
    };
    auto pgnorms = [&](std::vector<double> &pg) -> sr_status {
        lbf_pgnorm_kernel<<<nch, kLbThreads, 0, st>>>(chunks, x, g, ridx, loR, pgpart);
        std::vector<float> hp(nch);
        SR_CUDA(cudaMemcpyAsync(hp.data(), pgpart, sizeof(float) * nch, cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        pg.assign(nf, 0.0);
        for (int f = 0; f < nf; ++f)
            for (int c = c0[f]; c < c0[f + 1]; ++c) pg[f] = std::max(pg[f], (double)hp[c]);
        return SR_OK;
    };
    std::vector<double> fcur(nf), fl(nf);
    sr_status rs;
    auto eval = [&](const float *xv, float *gv, std::vector<double> &fv) -> sr_status {
        sr_status s2 = P.eval(xv, gv, losses);
        if (s2 != SR_OK) return s2;
        SR_CUDA(cudaMemcpyAsync(fv.data(), losses, sizeof(double) * nf, cudaMemcpyDeviceToHost, st));
        SR_CUDA(cudaStreamSynchronize(st));
        return SR_OK;
    };
    if ((rs = eval(x, g, fcur)) != SR_OK) return rs;
    const int H = cfg.max_iter + 1;
    if (f_hist)
        for (int f = 0; f < nf; ++f) {
            for (int i = 0; i < H; ++i) f_hist[(size_t)f * H + i] = NAN;
            f_hist[(size_t)f * H] = fcur[f];
        }
    std::vector<Memory> mem(nf);
    std::vector<int> it(nf, 0), evals(nf, 1), status(nf, SR_LBFGSB_MAX_ITER);
    std::vector<unsigned char> active(nf, cfg.max_iter > 0 ? 1 : 0);
    std::vector<double> pg(nf, 0.0);
    std::vector<FieldSearch> srch(nf);
    std::vector<DirArgs> hda(nf);
    std::vector<float> hx(nR), hg(nR), xcR_f(nR);
    std::vector<unsigned char> fix(nR);
    std::vector<unsigned char> ok(nf);
    const unsigned hw = std::thread::hardware_concurrency();
    const int threads = (int)std::min<unsigned>(hw ? hw : 1, 16);
    int rounds = 0;
    auto n_active = [&]() {
        int c = 0;
        for (int f = 0; f < nf; ++f) c += active[f];
        return c;
    };
    while (n_active() > 0) {
        if ((rs = pgnorms(pg)) != SR_OK) return rs;
        for (int f = 0; f < nf; ++f)
            if (active[f] && pg[f] <= cfg.pgtol) {
                status[f] = SR_LBFGSB_PGTOL;
                active[f] = 0;
            }
        if (n_active() == 0) break;
        // W^T g and g^T g per field
        std::vector<std::vector<uchar2>> lists(nf);
        int kmax = 0;
        for (int f = 0; f < nf; ++f) {
            const auto &sl = mem[f].slots;
            const int k = (int)sl.size();
            kmax = std::max(kmax, k);
            for (int j = 0; j < k; ++j) lists[f].push_back(make_uchar2(vY(sl[j]), VG));
            for (int j = 0; j < k; ++j) lists[f].push_back(make_uchar2(vS(sl[j]), VG));
            lists[f].push_back(make_uchar2(VG, VG));
        }
        std::vector<std::vector<double>> dv;
        if ((rs = segdots(lists, dv)) != SR_OK) return rs;
        // the bounded rows with each field's rows of W
        for (int f = 0; f < nf; ++f) {
            hda[f] = DirArgs{};
            hda[f].k = (int)mem[f].slots.size();
            for (int j = 0; j < hda[f].k; ++j) hda[f].slot[j] = mem[f].slots[j];
        }
        std::vector<float> hW((size_t)2 * kmax * nR);
        if (nR > 0) {
            SR_CUDA(cudaMemcpyAsync(dargs, hda.data(), sizeof(DirArgs) * nf, cudaMemcpyHostToDevice, st));
            lbf_gather_kernel<<<gR, 256, 0, st>>>(rsrc, rfid, nR, dargs, x, g, S, Y, n, gx, gg_, gW);
            SR_CUDA(cudaMemcpyAsync(hx.data(), gx, sizeof(float) * nR, cudaMemcpyDeviceToHost, st));
            SR_CUDA(cudaMemcpyAsync(hg.data(), gg_, sizeof(float) * nR, cudaMemcpyDeviceToHost, st));
            if (kmax) SR_CUDA(cudaMemcpyAsync(hW.data(), gW, sizeof(float) * 2 * kmax * nR, cudaMemcpyDeviceToHost, st));
            SR_CUDA(cudaStreamSynchronize(st));
        }
        // the host half per active field, in parallel over fields
        parallel_for(nf, threads, [&](int f) {
            ok[f] = 1;
            if (!active[f]) return;
            const int k = (int)mem[f].slots.size();
            std::vector<double> Wg(2 * k);
            for (int j = 0; j < k; ++j) {
                Wg[j] = dv[f][j];
                Wg[k + j] = mem[f].theta * dv[f][k + j];
            }
            Rows R;
            R.nR = r0[f + 1] - r0[f];
            R.x = hx.data() + r0[f];
            R.g = hg.data() + r0[f];
            R.lo = hlo.data() + r0[f];
            R.W = hW.data() + r0[f];
            R.stride = nR;
            ok[f] = cauchy_subspace(mem[f], Wg, dv[f][2 * k], R, hda[f], xcR_f.data() + r0[f], fix.data() + r0[f]) ? 1 : 0;
        });
        for (int f = 0; f < nf; ++f)
            if (active[f] && !ok[f]) {
                status[f] = SR_LBFGSB_LINE_SEARCH;
                active[f] = 0;
            }
        SR_CUDA(cudaMemcpyAsync(dargs, hda.data(), sizeof(DirArgs) * nf, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaMemcpyAsync(act, active.data(), nf, cudaMemcpyHostToDevice, st));
        if (nR > 0) {
            SR_CUDA(cudaMemcpyAsync(xcR, xcR_f.data(), sizeof(float) * nR, cudaMemcpyHostToDevice, st));
            SR_CUDA(cudaMemcpyAsync(fixR, fix.data(), nR, cudaMemcpyHostToDevice, st));
        }
        lbf_dir_kernel<<<gb, kLbThreads, 0, st>>>(dargs, act, fid, x, g, S, Y, n, ridx, xcR, fixR, d);
        // line searches along d, one batched evaluation per round
        std::vector<std::vector<uchar2>> ddl(nf, {make_uchar2(VD, VD), make_uchar2(VG, VD)});
        std::vector<std::vector<double>> dd;
        if ((rs = segdots(ddl, dd)) != SR_OK) return rs;
        for (int f = 0; f < nf; ++f) {
            srch[f] = FieldSearch{};
            if (!active[f]) continue;
            const double dn = std::sqrt(dd[f][0]), dphi0 = dd[f][1];
            if (dn == 0.0) {
                status[f] = SR_LBFGSB_PGTOL;
                active[f] = 0;
                continue;
            }
            if (!(dphi0 < 0.0)) {
                status[f] = SR_LBFGSB_LINE_SEARCH;
                active[f] = 0;
                continue;
            }
            FieldSearch &s = srch[f];
            s.searching = cfg.max_ls > 0;
            s.f0 = fcur[f];
            s.dphi0 = dphi0;
            s.f_prev = fcur[f];
            s.a = it[f] == 0 ? std::min(1.0, 1.0 / dn) : 1.0;
        }
        std::vector<float> ha(nf);
        std::vector<std::vector<uchar2>> gdl(nf, {make_uchar2(VGT, VD)});
        for (;;) {
            int nsearch = 0;
            for (int f = 0; f < nf; ++f) {
                nsearch += srch[f].searching;
                // searching: the next trial; found: the accepted step again (xt, gt keep it);
                // otherwise no move
                ha[f] = (srch[f].searching || srch[f].found) ? (float)srch[f].a : 0.f;
            }
            if (nsearch == 0) break;
            SR_CUDA(cudaMemcpyAsync(astep, ha.data(), sizeof(float) * nf, cudaMemcpyHostToDevice, st));
            lbf_axpy_kernel<<<gb, 256, 0, st>>>(x, d, astep, fid, n, xt);
            if ((rs = eval(xt, gt, fl)) != SR_OK) return rs;
            ++rounds;
            std::vector<std::vector<double>> gd;
            if ((rs = segdots(gdl, gd)) != SR_OK) return rs;
            for (int f = 0; f < nf; ++f)
                if (srch[f].searching) {
                    ++evals[f];
                    search_update(srch[f], fl[f], gd[f][0], cfg.max_ls);
                }
        }
        // every field that found a step: its candidate pair, the memory update and the step
        std::vector<int> hcol(nf, -1);
        for (int f = 0; f < nf; ++f) {
            if (!active[f]) continue;
            if (!srch[f].found) {
                status[f] = SR_LBFGSB_LINE_SEARCH;
                active[f] = 0;
                continue;
            }
            hcol[f] = free_column(mem[f]);
        }
        SR_CUDA(cudaMemcpyAsync(colv, hcol.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, st));
        lbf_pair_kernel<<<gb, 256, 0, st>>>(colv, fid, x, xt, g, gt, n, S, Y);
        std::vector<std::vector<uchar2>> pl(nf);
        for (int f = 0; f < nf; ++f) {
            if (hcol[f] < 0) continue;
            const unsigned char sc = vS(hcol[f]), yc = vY(hcol[f]);
            pl[f] = {make_uchar2(sc, yc), make_uchar2(yc, yc), make_uchar2(sc, sc)};
            for (int sj : mem[f].slots) {
                pl[f].push_back(make_uchar2(sc, vS(sj)));
                pl[f].push_back(make_uchar2(sc, vY(sj)));
                pl[f].push_back(make_uchar2(vS(sj), yc));
                pl[f].push_back(make_uchar2(yc, vY(sj)));
            }
        }
        std::vector<std::vector<double>> po;
        if ((rs = segdots(pl, po)) != SR_OK) return rs;
        lbf_accept_kernel<<<gb, 256, 0, st>>>(colv, fid, xt, gt, n, x, g);
        for (int f = 0; f < nf; ++f) {
            if (hcol[f] < 0) continue;
            push_pair(mem[f], m, hcol[f], po[f].data());
            const double fo = fcur[f];
            fcur[f] = srch[f].ft;
            ++it[f];
            if (f_hist) f_hist[(size_t)f * H + it[f]] = fcur[f];
            if ((fo - fcur[f]) / std::max({std::fabs(fo), std::fabs(fcur[f]), 1.0}) <=
                cfg.factr * 2.220446049250313e-16) {
                status[f] = SR_LBFGSB_FACTR;
                active[f] = 0;
            } else if (it[f] >= cfg.max_iter) {
                status[f] = SR_LBFGSB_MAX_ITER;
                active[f] = 0;
            }
        }
    }
    if ((rs = pgnorms(pg)) != SR_OK) return rs;
    SR_CUDA(cudaStreamSynchronize(st));
    if (info)
        for (int f = 0; f < nf; ++f) {
            info[f].iterations = it[f];
            info[f].evaluations = evals[f];
            info[f].status = status[f];
            info[f].f = fcur[f];
            info[f].pg_norm = pg[f];
        }
    if (rounds_out) *rounds_out = rounds;
    return SR_OK;
}

}  // namespace sr
