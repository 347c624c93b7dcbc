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
// Scratch per field (planes of F*F floats): c_1..c_{J-1} (planes 0..J-2), a pass buffer (J-1),
// and two T planes (J, J+1) used alternately; T_0 ends in plane J.
// One launch per pass covers every field of the table (fields deeper than a level skip it).
#include "common.cuh"
#include "kernels.cuh"

namespace sr {

__constant__ float kB3[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};

__device__ __forceinline__ int mirror_at(int t, int F) { return t < 0 ? -t : (t > F - 1 ? 2 * (F - 1) - t : t); }

__device__ __forceinline__ const float *c_plane(const FieldDev &fd, const float *params, int j) {
    return j == 0 ? params + fd.param_off : fd.starlet + (long long)(j - 1) * fd.F * fd.F;
}
__device__ __forceinline__ float *pass_plane(const FieldDev &fd) {
    return fd.starlet + (long long)(fd.J - 1) * fd.F * fd.F;
}
__device__ __forceinline__ float *t_plane(const FieldDev &fd, int j) {
    return fd.starlet + (long long)(fd.J + (j & 1)) * fd.F * fd.F;
}

// (H^T y)[n] along one axis: sum over taps m and over the mirror preimages of n.
__device__ __forceinline__ float adj_1d(const float *__restrict__ y, int n, int F, int step, int stride) {
    float acc = 0.f;
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

// Chunk items (256 pixels each) per block: their loads are in flight together, and the block's
// set-up (item, field) is paid once per 1024 pixels.
constexpr int kStarletChunks = 4;

// pass = 0: forward row pass; 1: forward column pass (+ detail plane, L1 partial);
//        2: adjoint column pass; 3: adjoint row pass (+ gamma).
__global__ void __launch_bounds__(256)
starlet_pass_kernel(const FieldDev *__restrict__ fields, const ChunkItem *__restrict__ chunks, int n_chunks,
                    const float *__restrict__ params, double *__restrict__ l1_part, int j, int pass) {
    __shared__ double s_red[kStarletChunks][8];
    const int step = 1 << j;
#pragma unroll
    for (int q = 0; q < kStarletChunks; ++q) {
        const int c = blockIdx.x * kStarletChunks + q;
        if (c >= n_chunks) break;  // uniform over the block
        const ChunkItem ch = chunks[c];
        const FieldDev &fd = fields[ch.field];
        if (j > fd.J - 2) continue;  // the field has no level j: the whole block skips this item
        const int F = fd.F;
        const int px = ch.start + threadIdx.x;
        const bool valid = px < F * F;
        const int y = valid ? px / F : 0, x = valid ? px - y * F : 0;
        const float lw = fd.lambda * fd.Wd[j];
        double l1 = 0.0;
        if (pass == 0) {
            if (valid) {
                const float *cj = c_plane(fd, params, j) + (long long)y * F;
                float acc = 0.f;
#pragma unroll
                for (int n = -2; n <= 2; ++n) acc += kB3[n + 2] * cj[mirror_at(x + n * step, F)];
                pass_plane(fd)[px] = acc;
            }
        } else if (pass == 1) {
            if (valid) {
                const float *tmp = pass_plane(fd);
                float acc = 0.f;
#pragma unroll
                for (int m = -2; m <= 2; ++m) acc += kB3[m + 2] * tmp[(long long)mirror_at(y + m * step, F) * F + x];
                float *cn = fd.starlet + (long long)j * F * F;  // c_{j+1}
                cn[px] = acc;
                const float wv = c_plane(fd, params, j)[px] - acc;
                l1 = (double)fabsf(wv);
            }
        } else if (pass == 2) {
            if (valid) {
                // v = T_{j+1} - gamma_{j+1}; tmp = Col^T v, gathered over the (up to three) rows k
                // whose mirrored taps land on row y
                const float *cj = c_plane(fd, params, j);
                const float *cn = fd.starlet + (long long)j * F * F;
                const bool has_t = (j + 1) < (fd.J - 1);
                const float *Tn = t_plane(fd, j + 1);
                auto v = [&](int k) {
                    const long long o = (long long)k * F + x;
                    const float wv = cj[o] - cn[o];
                    const float g = wv > 0.f ? lw : (wv < 0.f ? -lw : 0.f);
                    return (has_t ? Tn[o] : 0.f) - g;
                };
                float acc = 0.f;
#pragma unroll
                for (int m = -2; m <= 2; ++m) {
                    const float b = kB3[m + 2];
                    const int k1 = y - m * step;
                    if (k1 >= 0 && k1 < F) acc += b * v(k1);
                    const int k2 = -y - m * step;
                    if (y > 0 && k2 >= 0 && k2 < F) acc += b * v(k2);
                    const int k3 = 2 * (F - 1) - y - m * step;
                    if (y < F - 1 && k3 >= 0 && k3 < F) acc += b * v(k3);
                }
                pass_plane(fd)[px] = acc;
            }
        } else {
            if (valid) {
                const float *tmp = pass_plane(fd) + (long long)y * F;
                const float acc = adj_1d(tmp, x, F, step, 1);
                const float wv = c_plane(fd, params, j)[px] - fd.starlet[(long long)j * F * F + px];
                const float g = wv > 0.f ? lw : (wv < 0.f ? -lw : 0.f);
                t_plane(fd, j)[px] = g + acc;
            }
        }
        if (pass == 1) {
            // deterministic reduction of |w| over the item's 256 pixels
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l1 += __shfl_down_sync(0xffffffffu, l1, o);
            if ((threadIdx.x & 31) == 0) s_red[q][threadIdx.x >> 5] = l1;
        }
    }
    if (pass == 1) {
        __syncthreads();
        if (threadIdx.x < kStarletChunks) {
            const int c = blockIdx.x * kStarletChunks + threadIdx.x;
            if (c < n_chunks) {
                const ChunkItem ch = chunks[c];
                const FieldDev &fd = fields[ch.field];
                if (j <= fd.J - 2) {
                    double s = 0.0;
                    for (int i = 0; i < 8; ++i) s += s_red[threadIdx.x][i];
                    l1_part[fd.l1_slot + (long long)j * fd.n_chunks + ch.chunk] =
                        (double)fd.lambda * (double)fd.Wd[j] * s;
                }
            }
        }
    }
}

int launch_starlet(const FieldDev *fields, const ChunkItem *chunks, int n_chunks, int Jmax, const float *params,
                   double *l1_part, cudaStream_t st) {
    int n = 0;
    const int grid = (n_chunks + kStarletChunks - 1) / kStarletChunks;
    for (int j = 0; j <= Jmax - 2; ++j) {
        starlet_pass_kernel<<<grid, 256, 0, st>>>(fields, chunks, n_chunks, params, l1_part, j, 0);
        starlet_pass_kernel<<<grid, 256, 0, st>>>(fields, chunks, n_chunks, params, l1_part, j, 1);
        n += 2;
    }
    for (int j = Jmax - 2; j >= 0; --j) {
        starlet_pass_kernel<<<grid, 256, 0, st>>>(fields, chunks, n_chunks, params, l1_part, j, 2);
        starlet_pass_kernel<<<grid, 256, 0, st>>>(fields, chunks, n_chunks, params, l1_part, j, 3);
        n += 2;
    }
    return n;
}

}  // namespace sr
