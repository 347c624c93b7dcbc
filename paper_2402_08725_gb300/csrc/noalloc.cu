// Loss and gradient of one deconvolution field without any device allocation.
//
// The paper has no counterpart: this entry point serves callers that cannot call cudaMalloc
// (directly or through this library) — code running inside a device-memory pool fixed at start-up,
// a loop that must not block on the allocator, or a host runtime that owns all device memory.
// Every intermediate buffer of the evaluation (inverse-variance weights, folded PSF kernels,
// residual and adjoint images, partial sums, starlet planes and the work lists) is carved from one
// file-scope device array of SR_NOALLOC_SCRATCH_BYTES.  The kernels are the library's own
// (deconv.cu, starlet.cu, prep.cu); only where their scratch lives differs.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace sr {

// The scratch array: every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SR_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocMaxTiles = 16;  // N <= 256: at most 4 x 4 output tiles of 64 per epoch

// Device address of the array on each device, looked up once per device (host code cannot use the
// symbol's host-side name as a device address).  The mutex makes the first call on a device safe
// from several host threads: one of them does the set-up, the others wait for it.
static std::mutex g_scratch_mutex;
static void *g_scratch_addr[kNoallocMaxDevices];
static bool g_scratch_ready[kNoallocMaxDevices];

struct TileTemplate {
    int n;
    TileItem t[kNoallocMaxTiles];
};

struct WeightsArg {
    float w[kMaxScales];
};

// Writes the field description, the prior weights and the work lists into the scratch array.
__global__ void noalloc_setup_kernel(FieldDev fd, WeightsArg W, TileTemplate tt, FieldDev *fd_out, float *w_out,
                                     TileItem *items, int4 *ps, ChunkItem *chunks) {
    const long long n_items = (long long)fd.E * tt.n;
    const long long n_ps = (long long)fd.E * fd.M;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid == 0) *fd_out = fd;
    if (tid < kMaxScales) w_out[tid] = W.w[tid];
    for (long long i = tid; i < n_items; i += stride) {
        const int e = (int)(i / tt.n), k = (int)(i % tt.n);
        TileItem t = tt.t[k];
        t.epoch = e;
        t.slot = (int)i;
        items[i] = t;
    }
    for (long long i = tid; i < n_ps; i += stride) ps[i] = make_int4(0, (int)(i / fd.M), (int)(i % fd.M), 0);
    for (long long c = tid; c < fd.n_chunks; c += stride) chunks[c] = ChunkItem{0, (int)c * 256, (int)c};
}

static sr_status noalloc_fail(sr_status s, const char *msg) {
    set_error("%s", msg);
    return s;
}

struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += std::max<size_t>(n, 1) * sizeof(T);
        return at;
    }
};

}  // namespace sr

using namespace sr;

extern "C" sr_status sr_loss_and_grad_noalloc(const sr_problem_desc *desc, const float *d_dev, const float *sigma_dev,
                                              const float *psf_dev, const float *W_host, const float *params_dev,
                                              double *loss_dev, float *grad_dev, void *cuda_stream) {
    if (!desc || !d_dev || !sigma_dev || !psf_dev || !W_host || !params_dev || !loss_dev || !grad_dev)
        return noalloc_fail(SR_ERR_ARG, "sr_loss_and_grad_noalloc: NULL argument");
    const sr_problem_desc &D = *desc;
    if (D.kind != SR_DECONV) return noalloc_fail(SR_ERR_UNSUPPORTED, "sr_loss_and_grad_noalloc: deconvolution only");
    if (D.conv_mode == SR_CONV_PLAIN || D.conv_mode == SR_CONV_FFT)
        return noalloc_fail(SR_ERR_UNSUPPORTED, "sr_loss_and_grad_noalloc: the folded direct form only");
    if (D.n_epochs < 1 || D.data_n < 1 || D.data_n > 256 || D.supersampling < 1 || D.supersampling > 8 ||
        D.psf_k < 1 || D.psf_k > 511 || D.n_sources < 0 || D.n_sources > 64 || D.n_scales < 2 ||
        D.n_scales > kMaxScales || !(D.lambda >= 0.0))
        return noalloc_fail(SR_ERR_SHAPE, "sr_loss_and_grad_noalloc: sizes out of range (data_n must be <= 256)");
    const int N = D.data_n, f = D.supersampling, K = D.psf_k, E = D.n_epochs, M = D.n_sources, J = D.n_scales;
    const int F = f * N;
    if (2 * (1 << (J - 2)) > F - 1) return noalloc_fail(SR_ERR_SHAPE, "sr_loss_and_grad_noalloc: starlet wider than the grid");
    for (int j = 0; j < J - 1; ++j)
        if (!(W_host[j] >= 0.f)) return noalloc_fail(SR_ERR_NONFINITE, "sr_loss_and_grad_noalloc: weight < 0 or NaN");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // set-up, once per device, with that device current
    int dev = 0;
    SR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return noalloc_fail(SR_ERR_UNSUPPORTED, "device index too large");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ready[dev]) {
            void *ptr = nullptr;
            SR_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            int optin_dev = 0;
            SR_CUDA(cudaDeviceGetAttribute(&optin_dev, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            sr_status s = configure_tile_kernels(optin_dev - kTileStaticReserve, optin_dev - kTileStaticReserve);
            if (s != SR_OK) return s;
            g_scratch_addr[dev] = ptr;
            g_scratch_ready[dev] = true;
        }
        base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    }
    int optin = 0, n_sm = 0;
    SR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SR_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));

    // geometry of the folded kernels and of the output tiles (the same rules as a created problem)
    const int o = K / 2, t_lo = -o - f + 1, t_hi = K - 1 - o;
    const int tau_lo = t_lo >= 0 ? (t_lo + f - 1) / f : -((-t_lo) / f);
    const int tau_hi = (t_hi + f - 1) >= 0 ? (t_hi + f - 1) / f : -((-(t_hi + f - 1) + f - 1) / f);
    const int Tk = tau_hi - tau_lo + 1;
    const int nph = f * f;
    TileTemplate tt{};
    int smem_fwd = 0, smem_adj = 0;
    for (int y0 = 0; y0 < N; y0 += 64)
        for (int x0 = 0; x0 < N; x0 += 64) {
            TileItem t{};
            t.field = 0;
            t.y0 = (short)y0;
            t.x0 = (short)x0;
            t.h = (short)std::min(64, N - y0);
            t.w = (short)((std::min(64, N - x0) + kR - 1) / kR * kR);
            t.pg = choose_tile_pg(nph, t, Tk, optin - kTileStaticReserve);
            tt.t[tt.n++] = t;
            smem_fwd = std::max(smem_fwd, tile_smem_bytes(t, Tk, true));
            smem_adj = std::max(smem_adj, tile_smem_bytes(t, Tk, false));
        }
    const int n_chunks = (F * F + 255) / 256;
    const long long n_items = (long long)E * tt.n;
    Carve c;
    const size_t o_fd = c.take<FieldDev>(1), o_W = c.take<float>(kMaxScales), o_items = c.take<TileItem>(n_items);
    const size_t o_ps = c.take<int4>((size_t)E * M), o_chunks = c.take<ChunkItem>(n_chunks);
    const size_t o_cnt = c.take<int>(4), o_flag = c.take<int>(1);
    const size_t o_w = c.take<float>((size_t)E * N * N), o_kap = c.take<float>((size_t)E * nph * Tk * Tk);
    const size_t o_e = c.take<float>((size_t)E * N * N), o_g = c.take<float>((size_t)E * nph * N * N);
    const size_t o_chi = c.take<double>(n_items), o_se = c.take<double>(n_items);
    const size_t o_da = c.take<float>((size_t)E * M), o_du = c.take<float>(2 * (size_t)E * M);
    const size_t o_l1 = c.take<double>((size_t)(J - 1) * n_chunks), o_loss = c.take<double>(1);
    const size_t o_star = c.take<float>((size_t)(J + 2) * F * F);
    if (c.off > (size_t)SR_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg, "sr_loss_and_grad_noalloc: needs %zu bytes of scratch, the limit is %u", c.off,
                 (unsigned)SR_NOALLOC_SCRATCH_BYTES);
        return noalloc_fail(SR_ERR_SHAPE, msg);
    }

    if (smem_fwd > optin - kTileStaticReserve || smem_adj > optin - kTileStaticReserve)
        return noalloc_fail(SR_ERR_UNSUPPORTED, "sr_loss_and_grad_noalloc: PSF too large for shared memory");
    int bf = 1, ba = 1;
    sr_status s = occupancy_tile_kernels(smem_fwd, smem_adj, &bf, &ba);
    if (s != SR_OK) return s;
    const int grid_fwd = (int)std::max<long long>(1, std::min<long long>(n_items, (long long)std::max(bf, 1) * n_sm));
    const int grid_adj = (int)std::max<long long>(1, std::min<long long>(n_items, (long long)std::max(ba, 1) * n_sm));

    FieldDev fd{};
    fd.kind = SR_DECONV;
    fd.E = E;
    fd.N = N;
    fd.f = f;
    fd.K = K;
    fd.M = M;
    fd.J = J;
    fd.F = F;
    fd.Tk = Tk;
    fd.tau_lo = tau_lo;
    fd.n_tiles = tt.n;
    fd.lambda = (float)D.lambda;
    fd.Wd = reinterpret_cast<const float *>(base + o_W);
    fd.d = d_dev;
    fd.w = reinterpret_cast<const float *>(base + o_w);
    fd.kappa = reinterpret_cast<const float *>(base + o_kap);
    fd.starlet = reinterpret_cast<float *>(base + o_star);
    fd.n_chunks = n_chunks;
    WeightsArg wa{};
    for (int j = 0; j < J - 1; ++j) wa.w[j] = W_host[j];

    FieldDev *d_fd = reinterpret_cast<FieldDev *>(base + o_fd);
    TileItem *items = reinterpret_cast<TileItem *>(base + o_items);
    int4 *ps = reinterpret_cast<int4 *>(base + o_ps);
    ChunkItem *chunks = reinterpret_cast<ChunkItem *>(base + o_chunks);
    int *counters = reinterpret_cast<int *>(base + o_cnt);
    int *flag = reinterpret_cast<int *>(base + o_flag);
    float *w = reinterpret_cast<float *>(base + o_w);
    float *kappa = reinterpret_cast<float *>(base + o_kap);
    float *ebuf = reinterpret_cast<float *>(base + o_e);
    float *gbuf = reinterpret_cast<float *>(base + o_g);
    double *chi = reinterpret_cast<double *>(base + o_chi);
    double *se = reinterpret_cast<double *>(base + o_se);
    float *da = reinterpret_cast<float *>(base + o_da);
    float *du = reinterpret_cast<float *>(base + o_du);
    double *l1 = reinterpret_cast<double *>(base + o_l1);
    double *loss_field = reinterpret_cast<double *>(base + o_loss);

    const long long setup_work = std::max<long long>(std::max<long long>(n_items, (long long)E * M), n_chunks);
    const int setup_grid = (int)std::min<long long>((setup_work + 255) / 256 + 1, 4096);
    noalloc_setup_kernel<<<setup_grid, 256, 0, st>>>(fd, wa, tt, d_fd, reinterpret_cast<float *>(base + o_W), items,
                                                     ps, chunks);
    // the previous call's contents stay in the array: clear what the kernels accumulate into
    SR_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(int), st));
    SR_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    SR_CUDA(cudaMemsetAsync(da, 0, sizeof(float) * std::max<size_t>((size_t)E * M, 1), st));
    SR_CUDA(cudaMemsetAsync(du, 0, 2 * sizeof(float) * std::max<size_t>((size_t)E * M, 1), st));
    launch_inv_var(sigma_dev, w, (long long)E * N * N, flag, st);
    launch_kappa_prep(psf_dev, kappa, E, K, f, Tk, tau_lo, st);
    launch_fwd(d_fd, items, (int)n_items, counters, params_dev, ebuf, chi, se, grid_fwd, smem_fwd, st);
    launch_adj(d_fd, items, (int)n_items, counters + 1, ebuf, gbuf, grid_adj, smem_adj, st);
    if (E * M > 0) launch_psgrad(d_fd, ps, E * M, params_dev, gbuf, da, du, st);
    launch_starlet(d_fd, 1, F, starlet_forms_single(F, J, false), chunks, n_chunks, J, params_dev, l1, st);
    launch_hgrad(d_fd, chunks, n_chunks, gbuf, grad_dev, params_dev, st);
    launch_finalize(d_fd, 1, chi, se, l1, da, du, grad_dev, loss_field, loss_dev, st);
    // a sigma that is NaN or <= 0 has no inverse variance: the loss reports it as NaN
    launch_flag_to_nan(flag, loss_dev, st);
    SR_CUDA(cudaGetLastError());
    return SR_OK;
}
