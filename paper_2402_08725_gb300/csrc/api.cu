// Host side of the C ABI (include/starred.h): problem and batch objects, input validation,
// work-list construction, the evaluation launch sequence, and optimiser graphs.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "lbfgsb.cuh"

namespace sr {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

sr_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    cudaGetLastError();  // clear the sticky-free error state
    return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
}

static sr_status fail(sr_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

// Guard-band debug mode (environment variable SR_GUARD=1 when a buffer is allocated): every
// device buffer gets a tail of kGuardBytes filled with kGuardByte, and calls that return a host
// value verify that no tail was written (an overrun fails them with SR_ERR_STATE).
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;

static bool guard_mode() {
    const char *v = getenv("SR_GUARD");
    return v && v[0] == '1';
}

// Device allocations owned by one object, freed together.
struct DevArena {
    std::vector<void *> ptrs;
    std::vector<std::pair<unsigned char *, size_t>> guards;  // (tail start, bytes) when guarded
    template <typename T>
    sr_status alloc(T **p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        void *q = nullptr;
        const bool guard = guard_mode();
        const size_t bytes = n * sizeof(T);
        cudaError_t e = cudaMalloc(&q, bytes + (guard ? kGuardBytes : 0));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        ptrs.push_back(q);
        if (guard) {
            unsigned char *tail = static_cast<unsigned char *>(q) + bytes;
            e = cudaMemset(tail, kGuardByte, kGuardBytes);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
            guards.emplace_back(tail, kGuardBytes);
        }
        *p = static_cast<T *>(q);
        return SR_OK;
    }
    // SR_OK if every guard tail still holds the pattern (synchronous).
    sr_status check_guards() const {
        std::vector<unsigned char> buf(kGuardBytes);
        for (const auto &g : guards) {
            cudaError_t e = cudaMemcpy(buf.data(), g.first, g.second, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "guard check");
            for (size_t k = 0; k < g.second; ++k)
                if (buf[k] != kGuardByte) return fail(SR_ERR_STATE, "a device buffer was written past its end");
        }
        return SR_OK;
    }
    void release() {
        for (void *q : ptrs) cudaFree(q);
        ptrs.clear();
        guards.clear();
    }
    ~DevArena() { release(); }
};

static int g_smem_optin = -1;
static int g_num_sms = 0;
static int g_fft_smem_limit = 0;  // dynamic shared memory the transform kernels can take
static int g_fx_smem_limit = 0;   // ... and the per-epoch chunk kernel

// The limits are published (g_dev_ready, set last) only once every kernel is configured; host
// threads making their first calls together configure once, under the lock.
static std::mutex g_dev_mutex;
static std::atomic<bool> g_dev_ready{false};

static sr_status device_limits() {
    if (g_dev_ready.load(std::memory_order_acquire)) return SR_OK;
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (g_dev_ready.load(std::memory_order_relaxed)) return SR_OK;
    int dev = 0, optin = 0, sms = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // reserve the static shared memory of the tile kernels
    const int dyn = optin - kTileStaticReserve;
    sr_status s = configure_tile_kernels(dyn, dyn);
    if (s != SR_OK) return s;
    int fx = 0, fft = 0;
    s = configure_fft_pair(optin, &fx, &fft);
    if (s != SR_OK) return s;
    s = configure_fft_big(optin);
    if (s != SR_OK) return s;
    g_smem_optin = optin;
    g_num_sms = sms;
    g_fx_smem_limit = fx;
    g_fft_smem_limit = fft;
    g_dev_ready.store(true, std::memory_order_release);
    return SR_OK;
}

// Transform size for the frequency-domain form: the smallest listed L (the sizes the transform
// kernels are compiled for) that keeps the N x N output free of wrap-around,
// L >= N + max(tau_hi, -tau_lo), and holds the folded kernel, L >= Tk.
static bool fft_size(int N, int Tk, int tau_lo, int *L_out) {
    const int tau_hi = tau_lo + Tk - 1;
    const int L = fft_pair_next(std::max(N + std::max(tau_hi, -tau_lo), Tk));
    if (L == 0) return false;
    *L_out = L;
    return true;
}

// Polyphase extent of the folded kernels: tau in [tau_lo, tau_lo + Tk).
static void folded_extent(int K, int f, int *Tk, int *tau_lo) {
    const int o = K / 2;
    const int t_lo = -o - f + 1, t_hi = K - 1 - o;
    auto cdiv = [](int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); };
    auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int lo = cdiv(t_lo, f);
    const int hi = fdiv(t_hi + f - 1, f);
    *tau_lo = lo;
    *Tk = hi - lo + 1;
}

}  // namespace sr

using namespace sr;

// ------------------------------------------------------------------------------------------
// Execution plan: fields, work lists and scratch for one evaluation of one or many fields.
// ------------------------------------------------------------------------------------------
struct Plan {
    int kind = SR_DECONV;
    bool plain = false;
    int n_fields = 0;
    std::vector<FieldDev> h_fields;
    FieldDev *d_fields = nullptr;
    std::vector<size_t> param_off;
    size_t n_params = 0;
    // deconvolution work lists
    int n_items = 0;
    TileItem *d_items = nullptr;
    int *d_counters = nullptr;
    int smem_fwd = 0, smem_adj = 0, grid_fwd = 0, grid_adj = 0;
    int n_ps = 0;
    int4 *d_ps = nullptr;
    int n_chunks = 0;
    ChunkItem *d_chunks = nullptr;
    int Jmax = 0;
    int Fmax = 0;               // widest fine grid of the table (the starlet band grid)
    int starlet_forms = 0;  // 1 << starlet_field_form of every field (bands, tiles, comb bands)
    float *ebuf = nullptr, *gbuf = nullptr, *ps_da = nullptr, *ps_du = nullptr;
    double *chi_part = nullptr, *se_part = nullptr, *l1_part = nullptr, *losses = nullptr, *total = nullptr;
    // frequency-domain form
    int n_fft_items = 0, n_fft_fields = 0, max_pairs = 1, smem_fft = 0, smem_fx = 0, grid_fft = 0;
    int max_acc_points = 0;  // largest f^2 L (L/2 + 1) of the transform fields
    int chunk = kFftChunk, gp_cap = 0;  // the schedule the plan was built with (epochs per item, pair cap)
    int4 *d_fft_items = nullptr;
    int *d_fft_fields = nullptr;
    float2 *hhat = nullptr, *fft_acc = nullptr;
    // fields on the global-memory transforms: their table index and buffers
    std::vector<int> big_fields;
    std::vector<BigBuffers> big_buf;
    // fields whose channel moves with the epoch shifts: their shift gradients (2 per epoch)
    float *hs = nullptr;
    int hs_Emax = 0;
    // point-source prior (Eq. 11, third term): shadow entries of the fields that have it
    int n_sh = 0, sh_Fmax = 0, sh_Jmax = 0, sh_Mmax = 0, n_sh_chunks = 0;
    int sh_starlet_forms = 0;
    FieldDev *d_sh = nullptr;
    ChunkItem *d_sh_chunks = nullptr;
    float *pbar = nullptr, *abar = nullptr, *pts_g = nullptr;
    double *l1_pts = nullptr;
    // PSF
    PsfBuffers psf{};
    // plain form
    PlainBuffers plainb{};
    std::vector<const float *> s_raw;
    // optimiser
    uint8_t *d_group = nullptr;
    float *opt_m = nullptr, *opt_v = nullptr, *grad_int = nullptr, *params_int = nullptr;
    long long *d_t = nullptr;
    float *d_bc = nullptr;
    double **d_hist_ptr = nullptr;
    long long *d_hist_base = nullptr;
    cudaGraphExec_t graph = nullptr;
    const float *graph_params = nullptr;
    sr_optim_cfg graph_cfg{};
    int launches = 0;
    // kernel timing ring: events before the forward, between forward and adjoint, after the adjoint
    bool profiling = false;
    int prof_count = 0;
    std::vector<cudaEvent_t> prof_ev;
    DevArena arena;
    ~Plan() {
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    }
};

struct sr_problem {
    sr_problem_desc desc{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int F = 0, Tk = 0, tau_lo = 0;
    float *d = nullptr, *w = nullptr, *s = nullptr, *kappa = nullptr, *Wd = nullptr, *starlet = nullptr;
    float *psf_s = nullptr, *psf_tmp = nullptr, *psf_gs = nullptr;
    // frequency-domain form: transform geometry, twiddles, kernel spectra
    bool fft_ok = false;
    // the transform size is beyond shared memory: global-memory transforms (fft_big.cu), kernel
    // spectra in the transposed layout [E][f^2][L/2+1][L], and their set-up scratch
    bool fft_big = false;
    float2 *big_zb = nullptr, *big_zt = nullptr;
    // the extended channel moved with each epoch's shift (sr_set_translate_h; direct form only)
    bool translate_h = false;
    // rotated frames (sr_set_rotations; direct form only): per epoch (cos, sin) on the device
    bool rot_on = false;
    float *rot_dev = nullptr;
    std::vector<float> rot_host;
    // per-coefficient prior weights (sr_set_weight_map): [J-1][F][F] on the device
    bool wmap_on = false;
    float *wmap_dev = nullptr;
    int fft_L = 0;
    float2 *fft_tw = nullptr, *khat = nullptr;
    int *d_flag = nullptr;
    float W_host[kMaxScales] = {0};
    float Wd_host[kMaxScales] = {0};  // staging of the factors upload_weights writes
    // point-source prior: lambda_pts, its weights lambda_pts W_j (device, and the host copy they
    // are sent from) and the starlet scratch of the mean point-source image; pts_enabled once a
    // non-zero lambda_pts was set (the evaluation then carries the term)
    double lam_pts = 0.0;
    bool pts_enabled = false;
    float Wpts_host[kMaxScales] = {0};
    float *Wpts = nullptr, *pts_starlet = nullptr;
    bool has_data = false, has_noise = false, has_psfs = false, has_weights = false;
    bool pending_check = false;
    Plan *plan = nullptr;
    DevArena arena;
};

struct sr_batch {
    cudaStream_t stream = nullptr;
    std::vector<sr_problem *> probs;
    std::vector<char> pts_enabled;  // each problem's point-source prior state when the plan was built
    std::vector<char> translate;    // each problem's moved-channel state when the plan was built
    std::vector<char> rotate;       // each problem's rotated-frame state when the plan was built
    std::vector<char> wmap;         // each problem's weight-map state when the plan was built
    // batched input set-up (sr_batch_set_*), built at its first use
    DevArena bio_arena;
    BioEntry *bio_tab = nullptr;
    long long *bio_off_d = nullptr, *bio_off_s = nullptr, *bio_off_k = nullptr;
    long long bio_total_d = 0, bio_total_s = 0, bio_total_k = 0;
    bool bio_vec_d = false, bio_vec_s = false;  // every packed offset a multiple of 4 (float4 moves)
    int2 *bio_items = nullptr;
    std::vector<std::array<int, 3>> bio_ranges;  // (transform size L, first item, items) per size
    // host inputs are staged per kind (0 data, 1 noise, 2 PSFs) by copies on an internal stream:
    // a kind's copy waits until the launches that read its previous contents are done (free), the
    // batch's stream waits for the copy (copied), so copies overlap the set-up of other kinds
    float *bio_stage[3] = {nullptr, nullptr, nullptr};
    int *bio_flags = nullptr;   // the members' input flags gathered for one read-back
    bool bio_pending = false;   // a batched set-up call since the last check
    cudaStream_t bio_io = nullptr;
    cudaEvent_t bio_free[3] = {nullptr, nullptr, nullptr}, bio_copied[3] = {nullptr, nullptr, nullptr};
    ~sr_batch() {
        if (bio_io) cudaStreamDestroy(bio_io);
        for (int k = 0; k < 3; ++k) {
            if (bio_free[k]) cudaEventDestroy(bio_free[k]);
            if (bio_copied[k]) cudaEventDestroy(bio_copied[k]);
        }
    }
    Plan *plan = nullptr;
    int sched_chunk = 0, sched_gp = 0;  // requested schedule of the transform form (0: automatic)
};

// ------------------------------------------------------------------------------------------
static sr_status validate_desc(const sr_problem_desc *d) {
    if (!d) return fail(SR_ERR_ARG, "desc is NULL");
    if (d->kind != SR_DECONV && d->kind != SR_PSF) return fail(SR_ERR_ARG, "unknown kind %d", d->kind);
    if (d->n_epochs < 1 || d->n_epochs > 1000000) return fail(SR_ERR_SHAPE, "n_epochs %d out of range", d->n_epochs);
    if (d->data_n < 1 || d->data_n > 4096) return fail(SR_ERR_SHAPE, "data_n %d out of range", d->data_n);
    if (d->supersampling < 1 || d->supersampling > 8) return fail(SR_ERR_SHAPE, "supersampling %d out of range", d->supersampling);
    if (d->n_scales < 2 || d->n_scales > kMaxScales) return fail(SR_ERR_SHAPE, "n_scales %d out of range", d->n_scales);
    if (starlet_field_form(d->data_n * d->supersampling, d->n_scales) == 2)  // not reached for these bounds
        return fail(SR_ERR_SHAPE, "no starlet form for a %d-pixel grid with %d scales", d->data_n * d->supersampling,
                    d->n_scales);
    const int F = d->supersampling * d->data_n;
    if (2 * (1 << (d->n_scales - 2)) > F - 1)
        return fail(SR_ERR_SHAPE, "starlet with %d scales needs a grid wider than %d", d->n_scales, F);
    if (!(d->lambda >= 0.0) || !std::isfinite(d->lambda)) return fail(SR_ERR_ARG, "lambda must be finite and >= 0");
    if (d->kind == SR_DECONV) {
        if (d->psf_k < 1 || d->psf_k > 511) return fail(SR_ERR_SHAPE, "psf_k %d out of range", d->psf_k);
        if (d->n_sources < 0 || d->n_sources > 64) return fail(SR_ERR_SHAPE, "n_sources %d out of range", d->n_sources);
    }
    if (d->conv_mode < SR_CONV_AUTO || d->conv_mode > SR_CONV_FFT) return fail(SR_ERR_ARG, "unknown conv_mode");
    if (d->kind == SR_PSF && d->conv_mode == SR_CONV_FFT)
        return fail(SR_ERR_UNSUPPORTED, "the transform form exists for deconvolution problems only");
    if (d->kind == SR_PSF && d->conv_mode == SR_CONV_PLAIN)
        return fail(SR_ERR_UNSUPPORTED, "the plain form exists for deconvolution problems only");
    return SR_OK;
}

static size_t deconv_param_count(const sr_problem_desc &d) {
    const size_t F = (size_t)d.supersampling * d.data_n;
    const size_t E = d.n_epochs, M = d.n_sources;
    return F * F + E * M + 2 * M + 2 * E + E;
}
static size_t psf_param_count(const sr_problem_desc &d) {
    const size_t F = (size_t)d.supersampling * d.data_n;
    const size_t S = d.n_epochs;
    return F * F + 2 + S + 2 * S;
}
static size_t param_count(const sr_problem_desc &d) {
    return d.kind == SR_DECONV ? deconv_param_count(d) : psf_param_count(d);
}

static void layout_of(const sr_problem_desc &d, sr_layout *L) {
    memset(L, 0, sizeof *L);
    const size_t F = (size_t)d.supersampling * d.data_n;
    const size_t E = d.n_epochs;
    if (d.kind == SR_DECONV) {
        const size_t M = d.n_sources;
        const size_t cnt[5] = {F * F, E * M, 2 * M, 2 * E, E};
        size_t o = 0;
        for (int g = 0; g < 5; ++g) {
            L->offset[g] = o;
            L->count[g] = cnt[g];
            o += cnt[g];
        }
        L->n_groups = 5;
        L->total = o;
    } else {
        const size_t cnt[4] = {F * F, 2, E, 2 * E};
        size_t o = 0;
        for (int g = 0; g < 4; ++g) {
            L->offset[g] = o;
            L->count[g] = cnt[g];
            o += cnt[g];
        }
        L->n_groups = 4;
        L->total = o;
    }
}

static void fill_field_common(FieldDev &fd, sr_problem *p) {
    const sr_problem_desc &d = p->desc;
    memset(&fd, 0, sizeof fd);
    fd.kind = d.kind;
    fd.E = d.n_epochs;
    fd.N = d.data_n;
    fd.f = d.supersampling;
    fd.K = d.psf_k;
    fd.M = d.kind == SR_DECONV ? d.n_sources : 0;
    fd.J = d.n_scales;
    fd.F = p->F;
    fd.Tk = p->Tk;
    fd.tau_lo = p->tau_lo;
    fd.lambda = (float)d.lambda;
    fd.Wd = p->Wd;
    fd.d = p->d;
    fd.w = p->w;
    fd.kappa = p->kappa;
    fd.starlet = p->starlet;
    fd.psf_s = p->psf_s;
    fd.psf_tmp = p->psf_tmp;
    fd.psf_gs = p->psf_gs;
    fd.n_chunks = (fd.F * fd.F + 255) / 256;
    fd.mode = 0;
    fd.fft_L = p->fft_L;
    fd.fft_tw = p->fft_tw;
    fd.fft_khat = p->khat;
    fd.translate = p->translate_h ? 1 : 0;
    fd.hs_off = 0;
    fd.rot = p->rot_on ? reinterpret_cast<const float2 *>(p->rot_dev) : nullptr;
    fd.Wmap = p->wmap_on ? p->wmap_dev : nullptr;
}

// Epochs per work item of the frequency-domain form (one accumulator per item).

// Phase groups of a tile: the most phases at once that fit in the block's threads and in
// shared memory (one group always).
static int choose_pg(int nph, TileItem t, int Tk) {
    return choose_tile_pg(nph, t, Tk, g_smem_optin - kTileStaticReserve);
}

// ------------------------------------------------------------------------------------------
// Autotuner: which form (direct tiles or transforms) evaluates a field shape faster per epoch.
// ------------------------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::map<std::string, int> g_tune;  // "N,f,K,M" -> 0 direct, 1 transforms
static bool g_tune_loaded = false;

static std::string tune_key(const sr_problem_desc &d) {
    char buf[96];
    snprintf(buf, sizeof buf, "%d,%d,%d,%d", d.data_n, d.supersampling, d.psf_k, d.n_sources);
    return buf;
}

// Cache file named by SR_AUTOTUNE_CACHE: one JSON object {"N,f,K,M": mode, ...}.
static void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("SR_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    char key[96];
    int mode;
    int c;
    while ((c = fgetc(fp)) != EOF) {
        if (c != '"') continue;
        if (fscanf(fp, "%95[^\"]\": %d", key, &mode) == 2 && (mode == 0 || mode == 1)) g_tune[key] = mode;
    }
    fclose(fp);
}

static void tune_save() {
    const char *path = getenv("SR_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "w");
    if (!fp) return;
    fprintf(fp, "{");
    bool first = true;
    for (const auto &kv : g_tune) {
        fprintf(fp, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
        first = false;
    }
    fprintf(fp, "\n}\n");
    fclose(fp);
}

struct PlanOptions;
static sr_status time_form(sr_problem *p, int mode, float *ms);

static bool field_uses_fft(sr_problem *p, const PlanOptions &opt);

// Options of the single-field plans the autotuner times.
struct PlanOptions {
    int mode_override = -1;  // -1: the problem's own choice, 0: direct tiles, 1: transforms
    int epoch_limit = 0;     // > 0: evaluate only the first epochs
    int grid_limit = 0;      // > 0: at most this many blocks in the persistent kernels
    int chunk = 0;           // epochs per work item of the transform form (even, <= kFftChunk; 0: by rule)
    int gp_cap = 0;          // 1: one epoch pair per group in the transform form (0: the widest compiled)
};

static bool field_uses_fft(sr_problem *p, const PlanOptions &opt);

// Build the evaluation plan of `n` problems of the same kind.
static sr_status build_plan(Plan *pl, sr_problem *const *probs, int n, bool plain,
                            const PlanOptions &opt = PlanOptions()) {
    sr_status st = device_limits();
    if (st != SR_OK) return st;
    pl->kind = probs[0]->desc.kind;
    pl->plain = plain;
    pl->n_fields = n;
    pl->h_fields.resize(n);
    pl->param_off.resize(n);
    std::vector<TileItem> items;
    std::vector<int4> ps;
    std::vector<ChunkItem> chunks;
    std::vector<uint8_t> groups;
    long long ebuf = 0, gbuf = 0, tslot = 0, psslot = 0, l1slot = 0;
    size_t poff = 0;
    int Jmax = 0;
    int smem_fwd = 0, smem_adj = 0, smem_fft = 0, smem_fx = 0;
    std::vector<int4> fft_items;
    std::vector<int> fft_fields;
    long long hhat_len = 0, acc_len = 0;
    std::vector<FieldDev> sh;
    std::vector<ChunkItem> sh_chunks;
    long long pbar_len = 0, l1pts = 0, ptsslot = 0;
    long long hs_len = 0;
    // epochs per work item of the transform form: by default as many as keep at least two items per
    // SM (even, 2 .. kFftChunk), so that a single long field spreads over the GPU
    int chunk = opt.chunk;
    if (chunk <= 0) {
        long long ep = 0;
        for (int i = 0; i < n; ++i)
            if (probs[i]->fft_ok && !probs[i]->fft_big)
                ep += opt.epoch_limit > 0 ? std::min(probs[i]->desc.n_epochs, opt.epoch_limit) : probs[i]->desc.n_epochs;
        chunk = (int)std::min<long long>(kFftChunk, std::max<long long>(2, ep / (2LL * std::max(g_num_sms, 1)))) & ~1;
    }
    chunk = std::max(2, std::min(kFftChunk, chunk)) & ~1;
    pl->chunk = chunk;
    pl->gp_cap = opt.gp_cap;
    for (int i = 0; i < n; ++i) {
        sr_problem *p = probs[i];
        if (p->desc.kind != pl->kind) return fail(SR_ERR_ARG, "a batch mixes problem kinds");
        FieldDev &fd = pl->h_fields[i];
        fill_field_common(fd, p);
        if (opt.epoch_limit > 0) fd.E = std::min(fd.E, opt.epoch_limit);
        fd.param_off = (long long)poff;
        pl->param_off[i] = poff;
        const size_t np = param_count(p->desc);
        // optimiser groups
        sr_layout L;
        layout_of(p->desc, &L);
        const size_t g0 = groups.size();
        groups.resize(g0 + np);
        for (int g = 0; g < L.n_groups; ++g) {
            uint8_t gid = (uint8_t)g;
            if (pl->kind == SR_PSF) gid = (uint8_t)(g <= 1 ? g : g + 1);  // 0 b, 1 alpha, 2 beta, 3 a, 4 c
            for (size_t k = 0; k < L.count[g]; ++k) groups[g0 + L.offset[g] + k] = gid;
        }
        if (pl->kind == SR_PSF) groups[g0 + L.offset[1] + 1] = 2;  // beta
        poff += np;
        fd.ebuf_off = ebuf;
        ebuf += (long long)fd.E * fd.N * fd.N;
        fd.gbuf_off = gbuf;
        fd.l1_slot = l1slot;
        l1slot += (long long)(fd.J - 1) * fd.n_chunks;
        for (int c = 0; c < fd.n_chunks; ++c) chunks.push_back(ChunkItem{i, c * 256, c});
        Jmax = std::max(Jmax, fd.J);
        pl->Fmax = std::max(pl->Fmax, fd.F);
        pl->starlet_forms |= (1 << starlet_field_form(fd.F, fd.J)) | (fd.Wmap ? kStarletMapBit : 0);
        if (pl->kind == SR_DECONV && !plain && p->fft_big && field_uses_fft(p, opt)) {
            // global-memory transforms: one chi^2 / sum e slot per data row, the window adjoint
            // images of the point sources in gbuf, and per (epoch, source) gradient slots
            fd.mode = 2;
            fd.n_tiles = fd.N;
            fd.tile_slot = tslot;
            tslot += (long long)fd.E * fd.N;
            if (fd.M > 0) {
                fd.gbuf_off = gbuf;
                gbuf += (long long)fd.E * fd.f * fd.f * fd.N * fd.N;
            }
            fd.ps_slot = psslot;
            for (int e = 0; e < fd.E; ++e)
                for (int k = 0; k < fd.M; ++k) ps.push_back(make_int4(i, e, k, 0));
            psslot += (long long)fd.E * fd.M;
            pl->big_fields.push_back(i);
        } else if (pl->kind == SR_DECONV && !plain && field_uses_fft(p, opt)) {
            // frequency-domain form: chunks of consecutive epochs, one accumulator per chunk
            fd.mode = 1;
            fd.n_tiles = 1;
            fd.tile_slot = tslot;
            tslot += fd.E;
            fd.ps_slot = psslot;
            psslot += (long long)fd.E * fd.M;
            const int L = fd.fft_L, H = L / 2 + 1;
            const int nph = fd.f * fd.f;
            fd.fft_acc_off = acc_len;
            fd.fft_n_chunks = (fd.E + chunk - 1) / chunk;
            for (int c = 0; c < fd.fft_n_chunks; ++c)
                fft_items.push_back(make_int4(i, c * chunk, std::min(fd.E, (c + 1) * chunk), c));
            acc_len += (long long)fd.fft_n_chunks * nph * L * (H + 1);  // rows padded to H + 1
            fd.fft_hhat_off = hhat_len;
            hhat_len += (long long)nph * L * (H + 1);
            fft_fields.push_back(i);
            pl->max_pairs = std::max(pl->max_pairs, (nph + 1) / 2);
            pl->max_acc_points = std::max(pl->max_acc_points, nph * fd.fft_L * (fd.fft_L / 2 + 1));
            smem_fft = std::max(smem_fft, fft_pair_field_smem(L));
            // epoch pairs side by side: the widest group the kernel is compiled for at this size
            // (more than one pair only with at most one source) if its buffers fit, else one pair
            int G = fd.M <= 1 && opt.gp_cap != 1 ? fft_pair_gpmax(L) : 1;
            if (G > 1 && fft_pair_smem_bytes(L, fd.M, fd.f, G) > g_fx_smem_limit) G = 1;
            fd.fft_G = G;
            fd.fft_EB = fft_pair_zn(L);
            smem_fx = std::max(smem_fx, fft_pair_smem_bytes(L, fd.M, fd.f, G));
        } else if (pl->kind == SR_DECONV && !plain) {
            gbuf += (long long)fd.E * fd.f * fd.f * fd.N * fd.N;
            if (fd.translate) {
                fd.hs_off = hs_len;
                hs_len += 2LL * fd.E;
                pl->hs_Emax = std::max(pl->hs_Emax, fd.E);
            }
            const int nph = fd.f * fd.f;
            std::vector<TileItem> tiles;
            for (int y0 = 0; y0 < fd.N; y0 += 64)
                for (int x0 = 0; x0 < fd.N; x0 += 64) {
                    TileItem t{};
                    t.field = i;
                    t.y0 = (short)y0;
                    t.x0 = (short)x0;
                    t.h = (short)std::min(64, fd.N - y0);
                    t.w = (short)(((std::min(64, fd.N - x0)) + kR - 1) / kR * kR);
                    t.pg = choose_pg(nph, t, fd.Tk);
                    tiles.push_back(t);
                }
            fd.n_tiles = (int)tiles.size();
            fd.tile_slot = tslot;
            for (int e = 0; e < fd.E; ++e)
                for (int k = 0; k < fd.n_tiles; ++k) {
                    TileItem t = tiles[k];
                    t.epoch = e;
                    t.slot = (int)(tslot + (long long)e * fd.n_tiles + k);
                    items.push_back(t);
                    smem_fwd = std::max(smem_fwd, tile_smem_bytes(t, fd.Tk, true));
                    smem_adj = std::max(smem_adj, tile_smem_bytes(t, fd.Tk, false));
                }
            tslot += (long long)fd.E * fd.n_tiles;
            fd.ps_slot = psslot;
            for (int e = 0; e < fd.E; ++e)
                for (int k = 0; k < fd.M; ++k) ps.push_back(make_int4(i, e, k, 0));
            psslot += (long long)fd.E * fd.M;
        } else if (pl->kind == SR_DECONV) {
            if (fd.translate || fd.rot)
                return fail(SR_ERR_UNSUPPORTED, "the plain form does not move or rotate the extended channel");
            // plain form: per-epoch partials of the residual kernel, one slot per 256 data px
            const int nb = (fd.N * fd.N + 255) / 256;
            fd.n_tiles = nb;
            fd.tile_slot = tslot;
            tslot += (long long)fd.E * nb;
            fd.ps_slot = psslot;
            psslot += (long long)fd.E * fd.M;
        }
        if (pl->kind == SR_DECONV && p->pts_enabled && fd.M > 0) {
            if (plain) return fail(SR_ERR_UNSUPPORTED, "the plain form evaluates lambda_pts = 0 only");
            // shadow entry: the same field with c_0 = the mean point-source image
            FieldDev sd = fd;
            sd.lambda = 1.0f;
            sd.Wd = p->Wpts;
            sd.starlet = p->pts_starlet;
            sd.param_off = pbar_len;
            pbar_len += (long long)fd.F * fd.F;
            sd.l1_slot = l1pts;
            l1pts += (long long)(fd.J - 1) * fd.n_chunks;
            sd.ps_slot = ptsslot;
            ptsslot += fd.M;
            sd.pts = i + 1;
            fd.pts = (int)sh.size() + 1;
            for (int c = 0; c < fd.n_chunks; ++c) sh_chunks.push_back(ChunkItem{(int)sh.size(), c * 256, c});
            pl->sh_Fmax = std::max(pl->sh_Fmax, fd.F);
            pl->sh_Jmax = std::max(pl->sh_Jmax, fd.J);
            pl->sh_Mmax = std::max(pl->sh_Mmax, fd.M);
            pl->sh_starlet_forms |= (1 << starlet_field_form(fd.F, fd.J)) | (fd.Wmap ? kStarletMapBit : 0);
            sh.push_back(sd);
        }
    }
    if (tslot > 0x7fffffff) return fail(SR_ERR_SHAPE, "too many tiles");
    pl->Jmax = Jmax;
    pl->n_params = poff;
    DevArena &A = pl->arena;
    // sort the tile work list by decreasing cost so the persistent loops balance (LPT order)
    std::stable_sort(items.begin(), items.end(), [&](const TileItem &a, const TileItem &b) {
        const FieldDev &fa = pl->h_fields[a.field], &fb = pl->h_fields[b.field];
        const double ca = (double)a.h * a.w * fa.Tk * fa.Tk * fa.f * fa.f;
        const double cb = (double)b.h * b.w * fb.Tk * fb.Tk * fb.f * fb.f;
        return ca > cb;
    });
    std::stable_sort(fft_items.begin(), fft_items.end(), [&](const int4 &a, const int4 &b) {
        const FieldDev &fa = pl->h_fields[a.x], &fb = pl->h_fields[b.x];
        const double ca = (double)fa.fft_L * fa.fft_L * (2 + fa.f * fa.f) * (a.z - a.y);
        const double cb = (double)fb.fft_L * fb.fft_L * (2 + fb.f * fb.f) * (b.z - b.y);
        return ca > cb;
    });
    // the per-field transform kernels (h spectra, h gradient) take the costliest fields first, so
    // that their longest blocks start in the first wave; each block writes only its own field
    std::stable_sort(fft_fields.begin(), fft_fields.end(), [&](int a, int b) {
        const FieldDev &fa = pl->h_fields[a], &fb = pl->h_fields[b];
        const double ca = (double)fa.fft_L * fa.fft_L * (fa.fft_n_chunks + 1);
        const double cb = (double)fb.fft_L * fb.fft_L * (fb.fft_n_chunks + 1);
        return ca > cb;
    });
    {  // shorter comb-band blocks for tables too small to fill the GPU with 16-row ones
        std::vector<int> Fs, Js, sFs, sJs;
        for (int i = 0; i < n; ++i) {
            Fs.push_back(pl->h_fields[i].F);
            Js.push_back(pl->h_fields[i].J);
        }
        for (const FieldDev &sd : sh) {
            sFs.push_back(sd.F);
            sJs.push_back(sd.J);
        }
        pl->starlet_forms |= starlet_comb_rows_bits(Fs.data(), Js.data(), n, g_num_sms);
        if (!sh.empty()) pl->sh_starlet_forms |= starlet_comb_rows_bits(sFs.data(), sJs.data(), (int)sh.size(), g_num_sms);
    }
    pl->n_fft_items = (int)fft_items.size();
    pl->n_fft_fields = (int)fft_fields.size();
    pl->n_items = (int)items.size();
    pl->n_ps = (int)ps.size();
    pl->n_chunks = (int)chunks.size();
    if ((st = A.alloc(&pl->d_fields, n)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_items, items.size())) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_ps, ps.size())) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_chunks, chunks.size())) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_counters, 4)) != SR_OK) return st;
    if ((st = A.alloc(&pl->ebuf, (size_t)ebuf)) != SR_OK) return st;
    if ((st = A.alloc(&pl->gbuf, (size_t)gbuf)) != SR_OK) return st;
    if ((st = A.alloc(&pl->chi_part, (size_t)tslot)) != SR_OK) return st;
    if ((st = A.alloc(&pl->se_part, (size_t)tslot)) != SR_OK) return st;
    const size_t n_ps_slots = (size_t)std::max<long long>(psslot, 1);
    if ((st = A.alloc(&pl->ps_da, n_ps_slots)) != SR_OK) return st;
    if ((st = A.alloc(&pl->ps_du, 2 * n_ps_slots)) != SR_OK) return st;
    if ((st = A.alloc(&pl->l1_part, (size_t)l1slot)) != SR_OK) return st;
    if ((st = A.alloc(&pl->losses, (size_t)n)) != SR_OK) return st;
    if (hs_len > 0 && (st = A.alloc(&pl->hs, (size_t)hs_len)) != SR_OK) return st;
    if ((st = A.alloc(&pl->total, 1)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_group, poff)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_t, 1)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_bc, 2)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_hist_ptr, 1)) != SR_OK) return st;
    if ((st = A.alloc(&pl->d_hist_base, 1)) != SR_OK) return st;
    SR_CUDA(cudaMemset(pl->ps_da, 0, sizeof(float) * n_ps_slots));
    SR_CUDA(cudaMemset(pl->ps_du, 0, 2 * sizeof(float) * n_ps_slots));
    SR_CUDA(cudaMemset(pl->d_t, 0, sizeof(long long)));
    if (pl->kind == SR_PSF) {
        const FieldDev &fd = pl->h_fields[0];
        pl->psf.n_dchunks = (fd.N * fd.N + 255) / 256;
        pl->psf.ebuf = pl->ebuf;
        if ((st = A.alloc(&pl->psf.star_part, (size_t)fd.E * pl->psf.n_dchunks * 4)) != SR_OK) return st;
        if ((st = A.alloc(&pl->psf.ab_part, (size_t)fd.n_chunks * 2)) != SR_OK) return st;
    }
    if (plain) {
        const FieldDev &fd = pl->h_fields[0];
        const size_t F2 = (size_t)fd.F * fd.F;
        if ((st = A.alloc(&pl->plainb.fimg, F2)) != SR_OK) return st;
        if ((st = A.alloc(&pl->plainb.conv, F2)) != SR_OK) return st;
        if ((st = A.alloc(&pl->plainb.ey, F2)) != SR_OK) return st;
        if ((st = A.alloc(&pl->plainb.gsum, F2)) != SR_OK) return st;
        if ((st = A.alloc(&pl->plainb.gi, F2)) != SR_OK) return st;
        const int K = fd.K;
        const int T = 64;
        const long long need = (((long long)(T + K - 1) * ((T + K) | 1) + 3) / 4 * 4 + (long long)K * ((K + 3) & ~3)) * 4;
        if (need > g_smem_optin - kTileStaticReserve)
            return fail(SR_ERR_UNSUPPORTED, "plain form: PSF size %d needs %lld bytes of shared memory", K, need);
        if ((st = configure_plain_kernels(K)) != SR_OK) return st;
    }
    SR_CUDA(cudaMemcpy(pl->d_fields, pl->h_fields.data(), sizeof(FieldDev) * n, cudaMemcpyHostToDevice));
    if (!sh.empty()) {
        pl->n_sh = (int)sh.size();
        pl->n_sh_chunks = (int)sh_chunks.size();
        if ((st = A.alloc(&pl->d_sh, sh.size())) != SR_OK) return st;
        if ((st = A.alloc(&pl->d_sh_chunks, sh_chunks.size())) != SR_OK) return st;
        if ((st = A.alloc(&pl->pbar, (size_t)pbar_len)) != SR_OK) return st;
        if ((st = A.alloc(&pl->l1_pts, (size_t)l1pts)) != SR_OK) return st;
        if ((st = A.alloc(&pl->abar, (size_t)ptsslot)) != SR_OK) return st;
        if ((st = A.alloc(&pl->pts_g, 3 * (size_t)ptsslot)) != SR_OK) return st;
        SR_CUDA(cudaMemcpy(pl->d_sh, sh.data(), sizeof(FieldDev) * sh.size(), cudaMemcpyHostToDevice));
        SR_CUDA(cudaMemcpy(pl->d_sh_chunks, sh_chunks.data(), sizeof(ChunkItem) * sh_chunks.size(),
                           cudaMemcpyHostToDevice));
    }
    if (!items.empty()) SR_CUDA(cudaMemcpy(pl->d_items, items.data(), sizeof(TileItem) * items.size(), cudaMemcpyHostToDevice));
    if (!ps.empty()) SR_CUDA(cudaMemcpy(pl->d_ps, ps.data(), sizeof(int4) * ps.size(), cudaMemcpyHostToDevice));
    if (!chunks.empty()) SR_CUDA(cudaMemcpy(pl->d_chunks, chunks.data(), sizeof(ChunkItem) * chunks.size(), cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemcpy(pl->d_group, groups.data(), groups.size(), cudaMemcpyHostToDevice));
    if (pl->n_fft_items > 0) {
        if (smem_fft > g_fft_smem_limit || smem_fx > g_fx_smem_limit)
            return fail(SR_ERR_UNSUPPORTED, "transform form needs %d + %d bytes of shared memory", smem_fft, smem_fx);
        pl->smem_fft = smem_fft;
        pl->smem_fx = smem_fx;
        int bfft = 0;
        if ((st = occupancy_fft_pair(smem_fx, &bfft)) != SR_OK) return st;
        pl->grid_fft = std::max(1, std::min(pl->n_fft_items, std::max(bfft, 1) * g_num_sms));
        if (opt.grid_limit > 0) pl->grid_fft = std::min(pl->grid_fft, opt.grid_limit);
        if ((st = A.alloc(&pl->d_fft_items, fft_items.size())) != SR_OK) return st;
        if ((st = A.alloc(&pl->d_fft_fields, fft_fields.size())) != SR_OK) return st;
        if ((st = A.alloc(&pl->hhat, (size_t)hhat_len)) != SR_OK) return st;
        if ((st = A.alloc(&pl->fft_acc, (size_t)acc_len)) != SR_OK) return st;
        SR_CUDA(cudaMemcpy(pl->d_fft_items, fft_items.data(), sizeof(int4) * fft_items.size(), cudaMemcpyHostToDevice));
        SR_CUDA(cudaMemcpy(pl->d_fft_fields, fft_fields.data(), sizeof(int) * fft_fields.size(), cudaMemcpyHostToDevice));
    }
    for (int i : pl->big_fields) {
        const FieldDev &fd = pl->h_fields[i];
        const size_t L = fd.fft_L, H = L / 2 + 1, nph = (size_t)fd.f * fd.f, npr = (nph + 1) / 2;
        BigBuffers bb{};
        if ((st = A.alloc(&bb.zb, (size_t)fd.E * npr * fd.N * L)) != SR_OK) return st;
        if ((st = A.alloc(&bb.zt, (size_t)fd.E * npr * fd.N * L)) != SR_OK) return st;
        if ((st = A.alloc(&bb.fhat, (size_t)fd.E * nph * H * L)) != SR_OK) return st;
        if ((st = A.alloc(&bb.acc, (size_t)((fd.E + 1) / 2) * nph * H * L)) != SR_OK) return st;
        pl->big_buf.push_back(bb);
    }
    if (pl->kind == SR_DECONV && !plain && pl->n_items > 0) {
        const int limit = g_smem_optin - kTileStaticReserve;
        if (smem_fwd > limit || smem_adj > limit)
            return fail(SR_ERR_UNSUPPORTED, "PSF size needs %d bytes of shared memory per block (limit %d)",
                        std::max(smem_fwd, smem_adj), limit);
        pl->smem_fwd = smem_fwd;
        pl->smem_adj = smem_adj;
        int bf = 0, ba = 0;
        if ((st = occupancy_tile_kernels(smem_fwd, smem_adj, &bf, &ba)) != SR_OK) return st;
        bf = std::max(bf, 1);
        ba = std::max(ba, 1);
        pl->grid_fwd = std::max(1, std::min(pl->n_items, bf * g_num_sms));
        pl->grid_adj = std::max(1, std::min(pl->n_items, ba * g_num_sms));
        if (opt.grid_limit > 0) {
            pl->grid_fwd = std::min(pl->grid_fwd, opt.grid_limit);
            pl->grid_adj = std::min(pl->grid_adj, opt.grid_limit);
        }
    }
    return SR_OK;
}

// Enqueue one loss-and-gradient evaluation of the plan on `st`.
static int run_eval(Plan *pl, const float *params, float *grad, cudaStream_t st,
                    const std::vector<const float *> *s_raw) {
    int n = 0;
    if (pl->kind == SR_PSF) {
        n += launch_psf_eval(pl->d_fields, pl->h_fields[0], pl->d_chunks, pl->n_chunks, params, grad, pl->psf,
                             pl->l1_part, pl->losses, pl->total, st);
        return n;
    }
    if (pl->plain) {
        n += launch_plain_eval(pl->d_fields, pl->h_fields[0], (*s_raw)[0], pl->d_chunks, pl->n_chunks, params, grad,
                               pl->plainb, pl->ebuf, pl->chi_part, pl->se_part, pl->ps_da, pl->ps_du, pl->d_ps,
                               pl->l1_part, pl->losses, pl->total, st);
        return n;
    }
    cudaMemsetAsync(pl->d_counters, 0, 4 * sizeof(int), st);
    cudaEvent_t *ev = nullptr;
    if (pl->profiling && !pl->prof_ev.empty()) {
        const int ring = (int)pl->prof_ev.size() / 4;
        ev = &pl->prof_ev[4 * (pl->prof_count % ring)];
        ++pl->prof_count;
        cudaEventRecord(ev[0], st);
    }
    if (pl->n_items > 0) {
        launch_fwd(pl->d_fields, pl->d_items, pl->n_items, pl->d_counters, params, pl->ebuf, pl->chi_part,
                   pl->se_part, pl->grid_fwd, pl->smem_fwd, st);
        if (ev) cudaEventRecord(ev[1], st);
        launch_adj(pl->d_fields, pl->d_items, pl->n_items, pl->d_counters + 1, pl->ebuf, pl->gbuf, pl->grid_adj,
                   pl->smem_adj, st);
        n += 2;
    } else if (ev) {
        cudaEventRecord(ev[1], st);
    }
    if (ev) cudaEventRecord(ev[2], st);
    if (pl->n_fft_items > 0) {
        launch_fft_hhat_pair(pl->d_fields, pl->d_fft_fields, pl->n_fft_fields, pl->max_pairs, pl->smem_fft, params,
                             pl->hhat, st);
        launch_fft_chunks_pair(pl->d_fields, pl->d_fft_items, pl->n_fft_items, pl->d_counters + 2, params, pl->hhat,
                               pl->fft_acc, pl->chi_part, pl->se_part, pl->ps_da, pl->ps_du, pl->grid_fft, pl->smem_fx,
                               st);
        n += 2;
    }
    for (size_t b = 0; b < pl->big_fields.size(); ++b)
        n += launch_big_eval(pl->h_fields[pl->big_fields[b]], params, pl->big_buf[b], pl->ebuf, pl->gbuf, pl->chi_part,
                             pl->se_part, st);
    if (ev) cudaEventRecord(ev[3], st);
    if (pl->n_ps > 0) {
        launch_psgrad(pl->d_fields, pl->d_ps, pl->n_ps, params, pl->gbuf, pl->ps_da, pl->ps_du, st);
        ++n;
    }
    n += launch_starlet(pl->d_fields, pl->n_fields, pl->Fmax, pl->starlet_forms, pl->d_chunks, pl->n_chunks, pl->Jmax,
                        params, pl->l1_part, st);
    if (pl->n_items > 0) {
        launch_hgrad(pl->d_fields, pl->d_chunks, pl->n_chunks, pl->gbuf, grad, params, st);
        ++n;
        if (pl->hs) {
            launch_hshift_grad(pl->d_fields, pl->n_fields, pl->hs_Emax, params, pl->gbuf, pl->hs, st);
            ++n;
        }
    }
    if (pl->n_fft_items > 0) {
        n += launch_fft_hgrad_pair(pl->d_fields, pl->d_fft_fields, pl->n_fft_fields, pl->max_pairs, pl->smem_fft,
                                   pl->fft_acc, grad, pl->max_acc_points, g_num_sms, st);
    }
    for (size_t b = 0; b < pl->big_fields.size(); ++b)
        n += launch_big_hgrad(pl->h_fields[pl->big_fields[b]], pl->big_buf[b], grad, st);
    if (pl->n_sh > 0)
        n += launch_pts_prior(pl->d_sh, pl->d_fields, pl->n_sh, pl->sh_Fmax, pl->sh_Mmax, pl->sh_starlet_forms,
                              pl->d_sh_chunks, pl->n_sh_chunks, pl->sh_Jmax, params, pl->abar, pl->pbar, pl->l1_pts,
                              pl->pts_g, st);
    launch_finalize(pl->d_fields, pl->n_fields, pl->chi_part, pl->se_part, pl->l1_part, pl->ps_da, pl->ps_du, grad,
                    pl->losses, pl->total, st, pl->n_sh > 0 ? pl->d_sh : nullptr, pl->l1_pts, pl->pts_g, pl->hs);
    n += 2;
    return n;
}

// Time one loss-and-gradient evaluation of a problem in a given form on its first <= 16
// epochs with the persistent kernels on a single block: the cost per epoch on one SM, which is
// what decides a batch that fills the GPU either way.  Parameters are all zero (the kernels'
// work does not depend on the values).
static sr_status time_form(sr_problem *p, int mode, float *ms) {
    Plan pl;
    PlanOptions opt;
    opt.mode_override = mode;
    opt.epoch_limit = 16;
    opt.grid_limit = 1;
    sr_problem *arr[1] = {p};
    sr_status st = build_plan(&pl, arr, 1, false, opt);
    if (st != SR_OK) return st;
    float *params = nullptr, *grad = nullptr;
    if ((st = pl.arena.alloc(&params, pl.n_params)) != SR_OK) return st;
    if ((st = pl.arena.alloc(&grad, pl.n_params)) != SR_OK) return st;
    SR_CUDA(cudaMemsetAsync(params, 0, sizeof(float) * pl.n_params, p->stream));
    cudaEvent_t e0, e1;
    SR_CUDA(cudaEventCreate(&e0));
    SR_CUDA(cudaEventCreate(&e1));
    run_eval(&pl, params, grad, p->stream, nullptr);
    cudaEventRecord(e0, p->stream);
    for (int r = 0; r < 3; ++r) run_eval(&pl, params, grad, p->stream, nullptr);
    cudaEventRecord(e1, p->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    *ms = t / 3.f;
    return SR_OK;
}

static bool field_uses_fft(sr_problem *p, const PlanOptions &opt) {
    if (p->translate_h || p->rot_on) return false;  // the frame variants are evaluated in the direct form only
    if (opt.mode_override >= 0) return opt.mode_override == 1 && p->fft_ok;
    if (!p->fft_ok) return false;
    if (p->desc.conv_mode == SR_CONV_FFT) return true;
    if (p->desc.conv_mode != SR_CONV_AUTO) return false;
    if (p->fft_big) {
        // The one-block timing below does not apply to the global-memory transforms (they take the
        // whole GPU per launch); compare operation counts per epoch instead: the direct form's
        // 4 N^2 Tk^2 f^2 multiply-adds (model and adjoint) against about 50 L^2 log2(L^2) (f^2 + 4)
        // for the transforms and the spectral products.
        const double N = p->desc.data_n, f = p->desc.supersampling, Tk = p->Tk, L = p->fft_L;
        const double direct = 4.0 * N * N * Tk * Tk * f * f;
        const double transform = 50.0 * L * L * std::log2(L * L) * (f * f + 4.0);
        return transform < direct;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    const std::string key = tune_key(p->desc);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second == 1;
    float t_direct = 0.f, t_fft = 0.f;
    if (time_form(p, 0, &t_direct) != SR_OK || time_form(p, 1, &t_fft) != SR_OK) {
        cudaGetLastError();
        return true;  // the transform form fits; keep it when timing is not possible
    }
    const int mode = t_fft <= t_direct ? 1 : 0;
    g_tune[key] = mode;
    tune_save();
    return mode == 1;
}

static sr_status check_ready(sr_problem *p) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    if (!p->has_data) return fail(SR_ERR_STATE, "data not set");
    if (!p->has_noise) return fail(SR_ERR_STATE, "noise not set");
    if (p->desc.kind == SR_DECONV && !p->has_psfs) return fail(SR_ERR_STATE, "PSFs not set");
    if (!p->has_weights) return fail(SR_ERR_STATE, "weights not set");
    return SR_OK;
}

static sr_status check_flag(sr_problem *p) {
    int flag = 0;
    SR_CUDA(cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    SR_CUDA(cudaStreamSynchronize(p->stream));
    p->pending_check = false;
    if (flag) {
        SR_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream));
        return fail(SR_ERR_NONFINITE, "a non-finite value (or sigma <= 0) was found in the inputs");
    }
    return SR_OK;
}

static sr_status ensure_plan(sr_problem *p) {
    if (p->plan) return SR_OK;
    Plan *pl = new (std::nothrow) Plan();
    if (!pl) return fail(SR_ERR_OOM, "host allocation failed");
    sr_problem *arr[1] = {p};
    sr_status st = build_plan(pl, arr, 1, p->desc.kind == SR_DECONV && p->desc.conv_mode == SR_CONV_PLAIN);
    if (st != SR_OK) {
        delete pl;
        return st;
    }
    pl->s_raw.push_back(p->s);
    p->plan = pl;
    return SR_OK;
}

static sr_status ensure_opt_buffers(Plan *pl) {
    if (pl->opt_m) return SR_OK;
    sr_status st;
    if ((st = pl->arena.alloc(&pl->opt_m, pl->n_params)) != SR_OK) return st;
    if ((st = pl->arena.alloc(&pl->opt_v, pl->n_params)) != SR_OK) return st;
    if ((st = pl->arena.alloc(&pl->grad_int, pl->n_params)) != SR_OK) return st;
    SR_CUDA(cudaMemset(pl->opt_m, 0, sizeof(float) * pl->n_params));
    SR_CUDA(cudaMemset(pl->opt_v, 0, sizeof(float) * pl->n_params));
    SR_CUDA(cudaMemset(pl->d_t, 0, sizeof(long long)));
    return SR_OK;
}

static OptimArgs optim_args(const Plan *pl, const sr_optim_cfg &c) {
    OptimArgs a{};
    a.kind = c.kind;
    a.beta1 = c.beta1;
    a.beta2 = c.beta2;
    a.eps = c.eps;
    for (int g = 0; g < SR_MAX_GROUPS; ++g) {
        a.lr[g] = 0.f;
        a.lo[g] = -INFINITY;
    }
    if (pl->kind == SR_DECONV) {
        for (int g = 0; g < 5; ++g) a.lr[g] = c.lr[g];
        a.lo[1] = 0.f;  // a >= 0
    } else {
        a.lr[0] = c.lr[0];
        a.lr[1] = c.lr[1];
        a.lr[2] = c.lr[1];
        a.lr[3] = c.lr[2];
        a.lr[4] = c.lr[3];
        a.lo[1] = 1e-3f;   // alpha
        a.lo[2] = 1.001f;  // beta
        a.lo[3] = 0.f;     // a >= 0
    }
    return a;
}

__global__ void record_loss_kernel(const double *total, double *const *hist_ptr, const long long *t,
                                   const long long *base) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double *h = *hist_ptr;
        if (h) h[*t - *base] = *total;
    }
}

// n optimiser steps on plan `pl` (eager when the stream cannot be captured).
static sr_status run_steps(Plan *pl, cudaStream_t st, float *params, int n_steps, const sr_optim_cfg *cfg,
                           double *losses_dev, const std::vector<const float *> *s_raw) {
    sr_status s;
    if ((s = ensure_opt_buffers(pl)) != SR_OK) return s;
    const OptimArgs oa = optim_args(pl, *cfg);
    SR_CUDA(cudaMemcpyAsync(pl->d_hist_ptr, &losses_dev, sizeof(double *), cudaMemcpyHostToDevice, st));
    SR_CUDA(cudaMemcpyAsync(pl->d_hist_base, pl->d_t, sizeof(long long), cudaMemcpyDeviceToDevice, st));
    auto enqueue_one = [&](cudaStream_t s2) {
        pl->launches = run_eval(pl, params, pl->grad_int, s2, s_raw);
        record_loss_kernel<<<1, 32, 0, s2>>>(pl->total, pl->d_hist_ptr, pl->d_t, pl->d_hist_base);
        launch_opt_step((long long)pl->n_params, params, pl->grad_int, pl->opt_m, pl->opt_v, pl->d_group, oa, pl->d_t,
                        pl->d_bc, s2);
    };
    // the host copy of losses_dev must outlive the async copy above
    SR_CUDA(cudaStreamSynchronize(st));
    const bool capturable = st != nullptr && !pl->plain && !pl->profiling;
    if (!capturable) {
        for (int i = 0; i < n_steps; ++i) enqueue_one(st);
        SR_CUDA(cudaGetLastError());
        return SR_OK;
    }
    const bool same = pl->graph && pl->graph_params == params && memcmp(&pl->graph_cfg, cfg, sizeof *cfg) == 0;
    if (!same) {
        if (pl->graph) {
            cudaGraphExecDestroy(pl->graph);
            pl->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        SR_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        enqueue_one(st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&pl->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        pl->graph_params = params;
        pl->graph_cfg = *cfg;
    }
    for (int i = 0; i < n_steps; ++i) SR_CUDA(cudaGraphLaunch(pl->graph, st));
    return SR_OK;
}

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char *sr_last_error(void) { return g_err.c_str(); }
int sr_version(void) { return 1; }
int sr_build_arch(void) { return 103; }

sr_status sr_create_problem(const sr_problem_desc *desc, void *cuda_stream, sr_problem **out) {
    if (!out) return fail(SR_ERR_ARG, "out is NULL");
    *out = nullptr;
    sr_status st = validate_desc(desc);
    if (st != SR_OK) return st;
    sr_problem *p = new (std::nothrow) sr_problem();
    if (!p) return fail(SR_ERR_OOM, "host allocation failed");
    p->desc = *desc;
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&p->device);
    const sr_problem_desc &d = *desc;
    p->F = d.supersampling * d.data_n;
    const size_t E = d.n_epochs, N = d.data_n, F = p->F;
    DevArena &A = p->arena;
    auto bail = [&](sr_status s) {
        delete p;
        return s;
    };
    if ((st = A.alloc(&p->d, E * N * N)) != SR_OK) return bail(st);
    if ((st = A.alloc(&p->w, E * N * N)) != SR_OK) return bail(st);
    if ((st = A.alloc(&p->Wd, kMaxScales)) != SR_OK) return bail(st);
    if ((st = A.alloc(&p->starlet, (size_t)(d.n_scales + 2) * F * F)) != SR_OK) return bail(st);
    if ((st = A.alloc(&p->d_flag, 1)) != SR_OK) return bail(st);
    if (cudaMemset(p->d_flag, 0, sizeof(int)) != cudaSuccess) return bail(fail(SR_ERR_CUDA, "cudaMemset failed"));
    if (d.kind == SR_DECONV) {
        folded_extent(d.psf_k, d.supersampling, &p->Tk, &p->tau_lo);
        const size_t K = d.psf_k;
        if ((st = A.alloc(&p->s, E * K * K)) != SR_OK) return bail(st);
        if ((st = A.alloc(&p->kappa, E * d.supersampling * d.supersampling * (size_t)p->Tk * p->Tk)) != SR_OK)
            return bail(st);
        if (d.conv_mode == SR_CONV_FFT || d.conv_mode == SR_CONV_AUTO) {
            if ((st = device_limits()) != SR_OK) return bail(st);
            int L = 0;
            const bool ok = d.n_sources <= kFftMaxSources && fft_size(d.data_n, p->Tk, p->tau_lo, &L) &&
                            fft_pair_field_smem(L) <= g_fft_smem_limit && fft_pair_variant(L, d.n_sources, 1) &&
                            fft_pair_smem_bytes(L, d.n_sources, d.supersampling, 1) <= g_fx_smem_limit;
            // sizes beyond shared memory: the global-memory transforms of fft_big.cu
            const int tau_hi = p->tau_lo + p->Tk - 1;
            const int Lb = ok ? 0 : fft_big_next(std::max(d.data_n + std::max(tau_hi, -p->tau_lo), p->Tk));
            const bool big = !ok && Lb > 0 && fft_big_window_smem(p->Tk, d.supersampling) <= g_smem_optin - 2048;
            if (!ok && !big && d.conv_mode == SR_CONV_FFT)
                return bail(fail(SR_ERR_UNSUPPORTED, "the transform form does not fit this size"));
            if (big) {
                L = Lb;
                p->fft_big = true;
                const size_t H = L / 2 + 1, nph = (size_t)d.supersampling * d.supersampling, npr = (nph + 1) / 2;
                if ((st = A.alloc(&p->khat, E * nph * H * L)) != SR_OK) return bail(st);
                if ((st = A.alloc(&p->big_zb, E * npr * (size_t)p->Tk * L)) != SR_OK) return bail(st);
                if ((st = A.alloc(&p->big_zt, E * npr * (size_t)p->Tk * L)) != SR_OK) return bail(st);
            } else if (ok) {
                const size_t H = L / 2 + 1;
                // rows padded to H + 1 (even), so that column pairs are 16-byte aligned
                if ((st = A.alloc(&p->khat, E * d.supersampling * d.supersampling * (size_t)L * (H + 1))) != SR_OK)
                    return bail(st);
            }
            if (ok || big) {
                p->fft_ok = true;
                p->fft_L = L;
                if ((st = A.alloc(&p->fft_tw, (size_t)L)) != SR_OK) return bail(st);
                std::vector<float2> tw(L);
                for (int n = 0; n < L; ++n) {
                    const double a = -2.0 * M_PI * (double)n / (double)L;
                    tw[n] = make_float2((float)cos(a), (float)sin(a));
                }
                if (cudaMemcpy(p->fft_tw, tw.data(), sizeof(float2) * L, cudaMemcpyHostToDevice) != cudaSuccess)
                    return bail(fail(SR_ERR_CUDA, "twiddle upload failed"));
            }
        }
    } else {
        if ((st = A.alloc(&p->psf_s, F * F)) != SR_OK) return bail(st);
        if ((st = A.alloc(&p->psf_tmp, 3 * E * F * F)) != SR_OK) return bail(st);
        if ((st = A.alloc(&p->psf_gs, E * F * F)) != SR_OK) return bail(st);
    }
    *out = p;
    return SR_OK;
}

sr_status sr_destroy(sr_problem *p) {
    if (!p) return SR_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    delete p->plan;
    delete p;
    return SR_OK;
}

// The device address of page-locked host memory (cudaHostAlloc'ed or registered), else null.
static void *mapped_address(const void *host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Inputs in and results out of host memory.  From and to page-locked memory these are kernels
// reading or writing its mapped address: a copy-engine transfer that waits on earlier work of its
// stream (an evaluation, or kernels held back by a persistent launch of another stream) holds up,
// in the engine's queue, the staging copies that later set-up calls issue on the internal stream
// (measured: no overlap of the next step's inputs with this step's evaluation).
static sr_status params_in(float *dev, const float *host, size_t n, cudaStream_t st) {  // host -> device
    if (const float *m = static_cast<const float *>(mapped_address(host))) {
        launch_host_copy(m, dev, (long long)n, nullptr, nullptr, st);
        SR_CUDA(cudaGetLastError());
        return SR_OK;
    }
    SR_CUDA(cudaMemcpyAsync(dev, host, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    return SR_OK;
}

static sr_status results_out(float *grad_host, const float *grad_dev, size_t n, double *total_host,
                             const double *total_dev, cudaStream_t st) {
    float *mg = static_cast<float *>(mapped_address(grad_host));
    double *mt = static_cast<double *>(mapped_address(total_host));
    if (mg) {
        launch_host_copy(grad_dev, mg, (long long)n, mt ? total_dev : nullptr, mt, st);
        SR_CUDA(cudaGetLastError());
    } else {
        SR_CUDA(cudaMemcpyAsync(grad_host, grad_dev, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    }
    if (!mg || !mt) SR_CUDA(cudaMemcpyAsync(total_host, total_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    return SR_OK;
}

static sr_status copy_in(sr_problem *p, float *dst, const float *src, size_t n, int on_device) {
    if (!on_device) return params_in(dst, src, n, p->stream);
    SR_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    return SR_OK;
}

sr_status sr_set_data(sr_problem *p, const float *d, int on_device) {
    if (!p || !d) return fail(SR_ERR_ARG, "NULL argument");
    const size_t n = (size_t)p->desc.n_epochs * p->desc.data_n * p->desc.data_n;
    sr_status st = copy_in(p, p->d, d, n, on_device);
    if (st != SR_OK) return st;
    launch_check_finite(p->d, (long long)n, p->d_flag, p->stream);
    p->pending_check = true;
    p->has_data = true;
    return SR_OK;
}

sr_status sr_set_noise(sr_problem *p, const float *sigma, int on_device) {
    if (!p || !sigma) return fail(SR_ERR_ARG, "NULL argument");
    const size_t n = (size_t)p->desc.n_epochs * p->desc.data_n * p->desc.data_n;
    // sigma is staged in the weight buffer, then converted in place to w = 1/sigma^2
    sr_status st = copy_in(p, p->w, sigma, n, on_device);
    if (st != SR_OK) return st;
    launch_inv_var(p->w, p->w, (long long)n, p->d_flag, p->stream);
    p->pending_check = true;
    p->has_noise = true;
    return SR_OK;
}

sr_status sr_set_psfs(sr_problem *p, const float *s, int on_device) {
    if (!p || !s) return fail(SR_ERR_ARG, "NULL argument");
    if (p->desc.kind != SR_DECONV) return fail(SR_ERR_STATE, "set_psfs is for deconvolution problems");
    const sr_problem_desc &d = p->desc;
    const size_t n = (size_t)d.n_epochs * d.psf_k * d.psf_k;
    sr_status st = copy_in(p, p->s, s, n, on_device);
    if (st != SR_OK) return st;
    launch_check_finite(p->s, (long long)n, p->d_flag, p->stream);
    launch_kappa_prep(p->s, p->kappa, d.n_epochs, d.psf_k, d.supersampling, p->Tk, p->tau_lo, p->stream);
    if (p->khat) {
        FieldDev fd;
        fill_field_common(fd, p);
        if (p->fft_big) launch_big_kappa(fd, p->big_zb, p->big_zt, p->stream);
        else launch_fft_kappa_pair(fd, p->kappa, p->khat, p->stream);
    }
    SR_CUDA(cudaGetLastError());
    p->pending_check = true;
    p->has_psfs = true;
    return SR_OK;
}

// The per-scale factors the starlet kernels apply: W_j, or 1 with a per-coefficient map (which
// then carries the weights); the point-source shadow entry's lambda_pts times the same.
static sr_status upload_weights(sr_problem *p) {
    float w[kMaxScales];
    for (int j = 0; j < kMaxScales; ++j) w[j] = p->wmap_on ? 1.f : p->W_host[j];
    memcpy(p->Wd_host, w, sizeof w);
    SR_CUDA(cudaMemcpyAsync(p->Wd, p->Wd_host, sizeof w, cudaMemcpyHostToDevice, p->stream));
    if (p->Wpts) {
        for (int j = 0; j < kMaxScales; ++j) p->Wpts_host[j] = (float)(p->lam_pts * w[j]);
        SR_CUDA(cudaMemcpyAsync(p->Wpts, p->Wpts_host, sizeof p->Wpts_host, cudaMemcpyHostToDevice, p->stream));
    }
    return SR_OK;
}

sr_status sr_set_weights(sr_problem *p, const float *W) {
    if (!p || !W) return fail(SR_ERR_ARG, "NULL argument");
    const int nw = p->desc.n_scales - 1;
    for (int j = 0; j < nw; ++j)
        if (!(W[j] >= 0.f) || !std::isfinite(W[j])) return fail(SR_ERR_NONFINITE, "weight %d is not finite and >= 0", j);
    float tmp[kMaxScales] = {0};
    memcpy(tmp, W, sizeof(float) * nw);
    // staged through the problem's host copy so the caller's array may be reused at once
    memcpy(p->W_host, tmp, sizeof tmp);
    p->has_weights = true;
    return upload_weights(p);
}

sr_status sr_set_weight_map(sr_problem *p, const float *Wmap, int on_device) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    const bool on = Wmap != nullptr;
    sr_status st;
    if (on) {
        const size_t n = (size_t)(p->desc.n_scales - 1) * p->F * p->F;
        std::vector<float> h(n);
        if (on_device) {
            SR_CUDA(cudaMemcpyAsync(h.data(), Wmap, sizeof(float) * n, cudaMemcpyDeviceToHost, p->stream));
            SR_CUDA(cudaStreamSynchronize(p->stream));
        } else {
            memcpy(h.data(), Wmap, sizeof(float) * n);
        }
        for (size_t i = 0; i < n; ++i)
            if (!(h[i] >= 0.f) || !std::isfinite(h[i]))
                return fail(SR_ERR_NONFINITE, "weight-map entry %zu is not finite and >= 0", i);
        if (!p->wmap_dev && (st = p->arena.alloc(&p->wmap_dev, n)) != SR_OK) return st;
        SR_CUDA(cudaMemcpyAsync(p->wmap_dev, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice, p->stream));
        p->has_weights = true;
    }
    SR_CUDA(cudaStreamSynchronize(p->stream));
    if (on != p->wmap_on) {  // the next evaluation builds a plan with (or without) the map
        p->wmap_on = on;
        delete p->plan;
        p->plan = nullptr;
    }
    return upload_weights(p);
}

sr_status sr_set_translate_h(sr_problem *p, int enable) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    if (p->desc.kind != SR_DECONV) return fail(SR_ERR_STATE, "the moved channel belongs to deconvolution problems");
    const bool on = enable != 0;
    if (on && (p->desc.conv_mode == SR_CONV_FFT || p->desc.conv_mode == SR_CONV_PLAIN))
        return fail(SR_ERR_UNSUPPORTED, "moving the extended channel needs conv_mode AUTO or DIRECT");
    if (on == p->translate_h) return SR_OK;
    p->translate_h = on;
    if (p->plan) {  // the next evaluation builds a plan in the direct form (the optimiser state restarts)
        SR_CUDA(cudaStreamSynchronize(p->stream));
        delete p->plan;
        p->plan = nullptr;
    }
    return SR_OK;
}

sr_status sr_set_rotations(sr_problem *p, const double *theta) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    if (p->desc.kind != SR_DECONV) return fail(SR_ERR_STATE, "rotated frames belong to deconvolution problems");
    const bool on = theta != nullptr;
    const int E = p->desc.n_epochs;
    if (on) {
        if (p->desc.conv_mode == SR_CONV_FFT || p->desc.conv_mode == SR_CONV_PLAIN)
            return fail(SR_ERR_UNSUPPORTED, "rotated frames need conv_mode AUTO or DIRECT");
        for (int i = 0; i < E; ++i)
            if (!std::isfinite(theta[i])) return fail(SR_ERR_NONFINITE, "theta[%d] is not finite", i);
        sr_status st;
        if (!p->rot_dev && (st = p->arena.alloc(&p->rot_dev, 2 * (size_t)E)) != SR_OK) return st;
        p->rot_host.resize(2 * (size_t)E);
        for (int i = 0; i < E; ++i) {
            p->rot_host[2 * (size_t)i] = (float)std::cos(theta[i]);
            p->rot_host[2 * (size_t)i + 1] = (float)std::sin(theta[i]);
        }
        SR_CUDA(cudaMemcpyAsync(p->rot_dev, p->rot_host.data(), sizeof(float) * 2 * E, cudaMemcpyHostToDevice,
                                p->stream));
    }
    SR_CUDA(cudaStreamSynchronize(p->stream));
    if (on != p->rot_on) {  // the next evaluation builds a plan in the direct form (the optimiser restarts)
        p->rot_on = on;
        delete p->plan;
        p->plan = nullptr;
    }
    return SR_OK;
}

sr_status sr_set_lambda_pts(sr_problem *p, double lambda_pts) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    if (p->desc.kind != SR_DECONV) return fail(SR_ERR_STATE, "lambda_pts belongs to deconvolution problems");
    if (!(lambda_pts >= 0.0) || !std::isfinite(lambda_pts)) return fail(SR_ERR_ARG, "lambda_pts must be finite and >= 0");
    sr_status st;
    if (!p->Wpts && lambda_pts > 0.0) {
        // first non-zero value: the term's buffers, and a plan that carries it
        const size_t F2 = (size_t)p->F * p->F;
        if ((st = p->arena.alloc(&p->Wpts, kMaxScales)) != SR_OK) return st;
        if ((st = p->arena.alloc(&p->pts_starlet, (size_t)(p->desc.n_scales + 2) * F2)) != SR_OK) return st;
        p->pts_enabled = true;
        if (p->plan) {
            Plan *old = p->plan;
            SR_CUDA(cudaStreamSynchronize(p->stream));
            p->plan = nullptr;
            if ((st = ensure_plan(p)) != SR_OK) {
                p->plan = old;
                return st;
            }
            if (old->opt_m) {  // the optimiser's state carries over
                if ((st = ensure_opt_buffers(p->plan)) != SR_OK) return st;
                Plan *pl = p->plan;
                SR_CUDA(cudaMemcpyAsync(pl->opt_m, old->opt_m, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice,
                                        p->stream));
                SR_CUDA(cudaMemcpyAsync(pl->opt_v, old->opt_v, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice,
                                        p->stream));
                SR_CUDA(cudaMemcpyAsync(pl->d_t, old->d_t, sizeof(long long), cudaMemcpyDeviceToDevice, p->stream));
                SR_CUDA(cudaStreamSynchronize(p->stream));
            }
            delete old;
        }
    }
    p->lam_pts = lambda_pts;
    return upload_weights(p);
}

sr_status sr_psf_model(sr_problem *p, const float *params_dev, float *s_dev) {
    if (!p || !params_dev || !s_dev) return fail(SR_ERR_ARG, "NULL argument");
    if (p->desc.kind != SR_PSF) return fail(SR_ERR_STATE, "sr_psf_model needs a PSF problem");
    sr_status st;
    if ((st = ensure_plan(p)) != SR_OK) return st;
    launch_psf_model(p->plan->d_fields, p->F, params_dev, p->stream);
    SR_CUDA(cudaGetLastError());
    SR_CUDA(cudaMemcpyAsync(s_dev, p->psf_s, sizeof(float) * (size_t)p->F * p->F, cudaMemcpyDeviceToDevice,
                            p->stream));
    return SR_OK;
}

// The bounds of one problem's parameters at offset `off`: the lower bounds of the sr_step projection.
static void add_bounds(LbfgsbProblem &P, const sr_problem_desc &d, int F, long long off) {
    const long long r0 = off + (long long)F * F;
    if (d.kind == SR_DECONV) {
        const long long r1 = r0 + (long long)d.n_epochs * d.n_sources;
        P.ranges.push_back({r0, r1});
        P.lo.insert(P.lo.end(), (size_t)(r1 - r0), 0.0f);  // a >= 0
    } else {
        const long long r1 = r0 + 2 + d.n_epochs;
        P.ranges.push_back({r0, r1});
        P.lo.push_back(1e-3f);                                  // alpha
        P.lo.push_back(1.001f);                                 // beta
        P.lo.insert(P.lo.end(), (size_t)(r1 - r0 - 2), 0.0f);  // a >= 0
    }
}

static sr_status lbfgsb_config(const sr_lbfgsb_cfg *cfg, sr_lbfgsb_cfg *c) {
    *c = *cfg;
    if (c->m <= 0) c->m = kLbfgsMaxMemory;
    if (c->max_ls <= 0) c->max_ls = 20;
    if (c->m > kLbfgsMaxMemory || c->max_iter < 0 || !(c->pgtol >= 0.0) || !(c->factr >= 0.0))
        return fail(SR_ERR_ARG, "sr_lbfgsb: need m <= %d, max_iter >= 0, pgtol >= 0, factr >= 0", kLbfgsMaxMemory);
    return SR_OK;
}

sr_status sr_lbfgsb(sr_problem *p, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                    sr_lbfgsb_info *info) {
    if (!p || !params_dev || !cfg) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    sr_lbfgsb_cfg c;
    if ((st = lbfgsb_config(cfg, &c)) != SR_OK) return st;
    const sr_problem_desc &d = p->desc;
    LbfgsbProblem P;
    P.n = (long long)param_count(d);
    add_bounds(P, d, p->F, 0);
    P.eval = [p](const float *x, float *g, double *f) { return sr_loss_and_grad(p, x, f, nullptr, g); };
    return lbfgsb_run(P, params_dev, c, f_history, info, p->stream);
}

sr_status sr_estimate_lambda_pts(sr_problem *p, const float *params_dev, double *lambda_pts) {
    if (!p || !params_dev || !lambda_pts) return fail(SR_ERR_ARG, "NULL argument");
    if (p->desc.kind != SR_DECONV) return fail(SR_ERR_STATE, "lambda_pts belongs to deconvolution problems");
    if (!p->has_weights) return fail(SR_ERR_STATE, "weights not set");
    if (p->wmap_on) return fail(SR_ERR_UNSUPPORTED, "the App. C estimate takes per-scale weights (no weight map)");
    FieldDev fd;
    fill_field_common(fd, p);
    fd.param_off = 0;
    return pts_estimate(fd, params_dev, p->Wd, (float)p->desc.lambda, lambda_pts, p->stream);
}

size_t sr_param_count(const sr_problem *p) { return p ? param_count(p->desc) : 0; }

sr_status sr_param_layout(const sr_problem *p, sr_layout *out) {
    if (!p || !out) return fail(SR_ERR_ARG, "NULL argument");
    layout_of(p->desc, out);
    return SR_OK;
}

sr_status sr_loss_and_grad(sr_problem *p, const float *params_dev, double *loss_host, double *loss_dev,
                           float *grad_dev) {
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    if (!params_dev || !grad_dev) return fail(SR_ERR_ARG, "NULL params or grad");
    if ((st = ensure_plan(p)) != SR_OK) return st;
    Plan *pl = p->plan;
    pl->launches = run_eval(pl, params_dev, grad_dev, p->stream, &pl->s_raw);
    SR_CUDA(cudaGetLastError());
    if (loss_dev) SR_CUDA(cudaMemcpyAsync(loss_dev, pl->total, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    if (loss_host) {
        SR_CUDA(cudaMemcpyAsync(loss_host, pl->total, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        SR_CUDA(cudaStreamSynchronize(p->stream));
        if (p->pending_check && (st = check_flag(p)) != SR_OK) return st;
        if ((st = p->arena.check_guards()) != SR_OK || (st = pl->arena.check_guards()) != SR_OK) return st;
        if (!std::isfinite(*loss_host)) return fail(SR_ERR_NONFINITE, "the loss is not finite");
    }
    return SR_OK;
}

sr_status sr_loss(sr_problem *p, const float *params_dev, double *loss_host) {
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    if (!loss_host) return fail(SR_ERR_ARG, "loss_host is NULL");
    if ((st = ensure_plan(p)) != SR_OK) return st;
    if ((st = ensure_opt_buffers(p->plan)) != SR_OK) return st;
    return sr_loss_and_grad(p, params_dev, loss_host, nullptr, p->plan->grad_int);
}

sr_status sr_loss_and_grad_host(sr_problem *p, const float *params_host, double *loss_host, float *grad_host) {
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    if (!params_host || !loss_host || !grad_host) return fail(SR_ERR_ARG, "NULL argument");
    if ((st = ensure_plan(p)) != SR_OK) return st;
    Plan *pl = p->plan;
    if ((st = ensure_opt_buffers(pl)) != SR_OK) return st;
    if (!pl->params_int && (st = pl->arena.alloc(&pl->params_int, pl->n_params)) != SR_OK) return st;
    if ((st = params_in(pl->params_int, params_host, pl->n_params, p->stream)) != SR_OK) return st;
    if ((st = sr_loss_and_grad(p, pl->params_int, nullptr, nullptr, pl->grad_int)) != SR_OK) return st;
    if ((st = results_out(grad_host, pl->grad_int, pl->n_params, loss_host, pl->total, p->stream)) != SR_OK) return st;
    SR_CUDA(cudaStreamSynchronize(p->stream));
    if (p->pending_check && (st = check_flag(p)) != SR_OK) return st;
    if (!std::isfinite(*loss_host)) return fail(SR_ERR_NONFINITE, "the loss is not finite");
    return SR_OK;
}

sr_status sr_loss_and_grad_host_async(sr_problem *p, const float *params_host, double *loss_host, float *grad_host) {
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    if (!params_host || !loss_host || !grad_host) return fail(SR_ERR_ARG, "NULL argument");
    if ((st = ensure_plan(p)) != SR_OK) return st;
    Plan *pl = p->plan;
    if ((st = ensure_opt_buffers(pl)) != SR_OK) return st;
    if (!pl->params_int && (st = pl->arena.alloc(&pl->params_int, pl->n_params)) != SR_OK) return st;
    if ((st = params_in(pl->params_int, params_host, pl->n_params, p->stream)) != SR_OK) return st;
    if ((st = sr_loss_and_grad(p, pl->params_int, nullptr, nullptr, pl->grad_int)) != SR_OK) return st;
    return results_out(grad_host, pl->grad_int, pl->n_params, loss_host, pl->total, p->stream);
}

sr_status sr_sync(sr_problem *p) {
    if (!p) return fail(SR_ERR_ARG, "problem is NULL");
    SR_CUDA(cudaStreamSynchronize(p->stream));
    if (p->pending_check) return check_flag(p);
    return SR_OK;
}

sr_status sr_step(sr_problem *p, float *params_dev, int n_steps, const sr_optim_cfg *cfg, double *losses_dev,
                  double *last_loss_host) {
    sr_status st = check_ready(p);
    if (st != SR_OK) return st;
    if (!params_dev || !cfg || n_steps < 0) return fail(SR_ERR_ARG, "bad argument");
    if (cfg->kind != SR_ADABELIEF && cfg->kind != SR_ADAM) return fail(SR_ERR_ARG, "unknown optimiser");
    if ((st = ensure_plan(p)) != SR_OK) return st;
    if ((st = run_steps(p->plan, p->stream, params_dev, n_steps, cfg, losses_dev, &p->plan->s_raw)) != SR_OK) return st;
    if (last_loss_host) {
        SR_CUDA(cudaMemcpyAsync(last_loss_host, p->plan->total, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        SR_CUDA(cudaStreamSynchronize(p->stream));
        if (p->pending_check && (st = check_flag(p)) != SR_OK) return st;
    }
    return SR_OK;
}

sr_status sr_reset_optimizer(sr_problem *p) {
    if (!p) return fail(SR_ERR_ARG, "NULL problem");
    sr_status st;
    if ((st = ensure_plan(p)) != SR_OK) return st;
    if ((st = ensure_opt_buffers(p->plan)) != SR_OK) return st;
    Plan *pl = p->plan;
    SR_CUDA(cudaMemsetAsync(pl->opt_m, 0, sizeof(float) * pl->n_params, p->stream));
    SR_CUDA(cudaMemsetAsync(pl->opt_v, 0, sizeof(float) * pl->n_params, p->stream));
    SR_CUDA(cudaMemsetAsync(pl->d_t, 0, sizeof(long long), p->stream));
    return SR_OK;
}

sr_status sr_get_state(sr_problem *p, float *m_dev, float *v_dev, int64_t *t) {
    if (!p || !m_dev || !v_dev || !t) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    if ((st = ensure_plan(p)) != SR_OK) return st;
    if ((st = ensure_opt_buffers(p->plan)) != SR_OK) return st;
    Plan *pl = p->plan;
    long long tv = 0;
    SR_CUDA(cudaMemcpyAsync(m_dev, pl->opt_m, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice, p->stream));
    SR_CUDA(cudaMemcpyAsync(v_dev, pl->opt_v, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice, p->stream));
    SR_CUDA(cudaMemcpyAsync(&tv, pl->d_t, sizeof(long long), cudaMemcpyDeviceToHost, p->stream));
    SR_CUDA(cudaStreamSynchronize(p->stream));
    *t = (int64_t)tv;
    return SR_OK;
}

sr_status sr_set_state(sr_problem *p, const float *m_dev, const float *v_dev, int64_t t) {
    if (!p || !m_dev || !v_dev || t < 0) return fail(SR_ERR_ARG, "bad argument");
    sr_status st;
    if ((st = ensure_plan(p)) != SR_OK) return st;
    if ((st = ensure_opt_buffers(p->plan)) != SR_OK) return st;
    Plan *pl = p->plan;
    long long tv = (long long)t;
    SR_CUDA(cudaMemcpyAsync(pl->opt_m, m_dev, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice, p->stream));
    SR_CUDA(cudaMemcpyAsync(pl->opt_v, v_dev, sizeof(float) * pl->n_params, cudaMemcpyDeviceToDevice, p->stream));
    SR_CUDA(cudaMemcpyAsync(pl->d_t, &tv, sizeof(long long), cudaMemcpyHostToDevice, p->stream));
    SR_CUDA(cudaStreamSynchronize(p->stream));
    return SR_OK;
}

int sr_launches_per_eval(const sr_problem *p) { return (p && p->plan) ? p->plan->launches : 0; }

// --- batches ------------------------------------------------------------------------------

sr_status sr_batch_create(sr_problem *const *problems, int n, void *cuda_stream, sr_batch **out) {
    if (!out) return fail(SR_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!problems || n < 1) return fail(SR_ERR_ARG, "empty batch");
    if (n > 65535) return fail(SR_ERR_ARG, "%d fields: a batch holds at most 65535", n);
    for (int i = 0; i < n; ++i) {
        sr_status st = check_ready(problems[i]);
        if (st != SR_OK) return st;
        if (problems[i]->desc.kind != SR_DECONV)
            return fail(SR_ERR_UNSUPPORTED, "batches hold deconvolution problems (field %d is a PSF fit)", i);
    }
    sr_batch *b = new (std::nothrow) sr_batch();
    if (!b) return fail(SR_ERR_OOM, "host allocation failed");
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->probs.assign(problems, problems + n);
    for (int i = 0; i < n; ++i) {
        b->pts_enabled.push_back(problems[i]->pts_enabled ? 1 : 0);
        b->translate.push_back(problems[i]->translate_h ? 1 : 0);
        b->rotate.push_back(problems[i]->rot_on ? 1 : 0);
        b->wmap.push_back(problems[i]->wmap_on ? 1 : 0);
    }
    b->plan = new (std::nothrow) Plan();
    if (!b->plan) {
        delete b;
        return fail(SR_ERR_OOM, "host allocation failed");
    }
    sr_status st = build_plan(b->plan, problems, n, false);
    if (st != SR_OK) {
        delete b->plan;
        delete b;
        return st;
    }
    *out = b;
    return SR_OK;
}

// Rebuilds the batch's plan with a schedule of the transform form (0: automatic).
static sr_status batch_replan(sr_batch *b, int chunk, int gp) {
    if (b->stream) SR_CUDA(cudaStreamSynchronize(b->stream));
    else SR_CUDA(cudaDeviceSynchronize());
    Plan *pl = new (std::nothrow) Plan();
    if (!pl) return fail(SR_ERR_OOM, "host allocation failed");
    PlanOptions opt;
    opt.chunk = chunk;
    opt.gp_cap = gp;
    sr_status st = build_plan(pl, b->probs.data(), (int)b->probs.size(), false, opt);
    if (st != SR_OK) {
        delete pl;
        return st;
    }
    delete b->plan;
    b->plan = pl;
    b->sched_chunk = chunk;
    b->sched_gp = gp;
    return SR_OK;
}

sr_status sr_batch_set_schedule(sr_batch *b, int epochs_per_item, int pairs_per_group) {
    if (!b) return fail(SR_ERR_ARG, "NULL batch");
    if (epochs_per_item < 0 || epochs_per_item > kFftChunk || (epochs_per_item & 1) ||
        (epochs_per_item > 0 && epochs_per_item < 2))
        return fail(SR_ERR_ARG, "epochs per item must be 0 (automatic) or even in 2..%d", kFftChunk);
    if (pairs_per_group != 0 && pairs_per_group != 1)
        return fail(SR_ERR_ARG, "pairs per group must be 0 (the widest compiled) or 1");
    return batch_replan(b, epochs_per_item, pairs_per_group);
}

sr_status sr_batch_get_schedule(const sr_batch *b, int *epochs_per_item, int *pairs_per_group) {
    if (!b || !epochs_per_item || !pairs_per_group) return fail(SR_ERR_ARG, "NULL argument");
    *epochs_per_item = b->plan->chunk;
    *pairs_per_group = b->plan->gp_cap;
    return SR_OK;
}

// Key of a batch's fields for the schedule cache: FNV-1a over each field's (N, E, f, K, M, form).
static std::string schedule_key(const sr_batch *b) {
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&](long long v) {
        for (int k = 0; k < 8; ++k) {
            h ^= (unsigned long long)((v >> (8 * k)) & 0xff);
            h *= 1099511628211ULL;
        }
    };
    for (size_t i = 0; i < b->probs.size(); ++i) {
        const sr_problem_desc &d = b->probs[i]->desc;
        mix(d.data_n);
        mix(d.n_epochs);
        mix(d.supersampling);
        mix(d.psf_k);
        mix(d.n_sources);
        mix(b->plan->h_fields[i].mode);
    }
    char buf[64];
    snprintf(buf, sizeof buf, "schedule:%016llx", h);
    return buf;
}

sr_status sr_batch_tune_schedule(sr_batch *b, int *epochs_per_item, int *pairs_per_group, float *ms_per_eval) {
    if (!b) return fail(SR_ERR_ARG, "NULL batch");
    sr_status st;
    const std::string key = schedule_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            const int c = it->second & 0xff, g = (it->second >> 8) & 0xff;
            if ((st = batch_replan(b, c, g)) != SR_OK) return st;
            if (epochs_per_item) *epochs_per_item = b->plan->chunk;
            if (pairs_per_group) *pairs_per_group = b->plan->gp_cap;
            if (ms_per_eval) *ms_per_eval = -1.f;  // from the cache, not timed
            return SR_OK;
        }
    }
    // time each candidate on zero parameters: one evaluation to warm up, then three
    float best_ms = 0.f;
    int best_c = 0, best_g = 0;
    cudaStream_t s = b->stream;
    for (int c : {2, 4, 8, 16})
        for (int g : {0, 1}) {
            if ((st = batch_replan(b, c, g)) != SR_OK) return st;
            Plan *pl = b->plan;
            if (pl->n_fft_items == 0 && (c != 2 || g != 0)) continue;  // nothing to schedule
            float *params = nullptr, *grad = nullptr;
            if ((st = pl->arena.alloc(&params, pl->n_params)) != SR_OK) return st;
            if ((st = pl->arena.alloc(&grad, pl->n_params)) != SR_OK) return st;
            SR_CUDA(cudaMemsetAsync(params, 0, sizeof(float) * pl->n_params, s));
            cudaEvent_t e0, e1;
            SR_CUDA(cudaEventCreate(&e0));
            SR_CUDA(cudaEventCreate(&e1));
            run_eval(pl, params, grad, s, nullptr);
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) run_eval(pl, params, grad, s, nullptr);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (e != cudaSuccess) return cuda_fail(e, "schedule timing");
            t /= 3.f;
            if (best_c == 0 || t < best_ms) {
                best_ms = t;
                best_c = c;
                best_g = g;
            }
        }
    if ((st = batch_replan(b, best_c, best_g)) != SR_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune[key] = best_c | (best_g << 8);
        tune_save();
    }
    if (epochs_per_item) *epochs_per_item = best_c;
    if (pairs_per_group) *pairs_per_group = best_g;
    if (ms_per_eval) *ms_per_eval = best_ms;
    return SR_OK;
}

sr_status sr_batch_destroy(sr_batch *b) {
    if (!b) return SR_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    delete b->plan;
    delete b;
    return SR_OK;
}

size_t sr_batch_param_count(const sr_batch *b) { return b ? b->plan->n_params : 0; }

sr_status sr_batch_param_offset(const sr_batch *b, int i, size_t *offset) {
    if (!b || !offset || i < 0 || i >= (int)b->probs.size()) return fail(SR_ERR_ARG, "bad argument");
    *offset = b->plan->param_off[i];
    return SR_OK;
}

// A problem whose point-source prior was switched on after the batch was built is not in the
// batch's plan: the batch must be re-created.
static sr_status batch_pts_check(const sr_batch *b) {
    for (size_t i = 0; i < b->probs.size(); ++i) {
        if ((b->probs[i]->pts_enabled ? 1 : 0) != b->pts_enabled[i])
            return fail(SR_ERR_STATE, "field %zu got a non-zero lambda_pts after sr_batch_create: re-create the batch", i);
        if ((b->probs[i]->translate_h ? 1 : 0) != b->translate[i])
            return fail(SR_ERR_STATE, "field %zu changed sr_set_translate_h after sr_batch_create: re-create the batch", i);
        if ((b->probs[i]->wmap_on ? 1 : 0) != b->wmap[i])
            return fail(SR_ERR_STATE, "field %zu set or cleared its weight map after sr_batch_create: re-create the batch",
                        i);
        if ((b->probs[i]->rot_on ? 1 : 0) != b->rotate[i])
            return fail(SR_ERR_STATE, "field %zu turned its rotations on or off after sr_batch_create: re-create the batch",
                        i);
    }
    return SR_OK;
}

static sr_status batch_check(sr_batch *b) {
    if (sr_status st = batch_pts_check(b)) return st;
    for (sr_problem *p : b->probs) {
        if (p->pending_check) {
            sr_status st = check_flag(p);
            if (st != SR_OK) return st;
        }
    }
    if (b->bio_pending) {
        // after batched set-up every flag write is ordered on the batch's stream (the members' own
        // pending set-up was synchronised just above): one gather
        const int n = (int)b->probs.size();
        std::vector<int> fl(n);
        launch_bio_flags(b->bio_tab, n, b->bio_flags, b->stream);
        SR_CUDA(cudaMemcpyAsync(fl.data(), b->bio_flags, sizeof(int) * n, cudaMemcpyDeviceToHost, b->stream));
        SR_CUDA(cudaStreamSynchronize(b->stream));
        b->bio_pending = false;
        for (int i = 0; i < n; ++i)
            if (fl[i]) return fail(SR_ERR_NONFINITE, "a non-finite value (or sigma <= 0) was found in the inputs of field %d", i);
    }
    return SR_OK;
}

sr_status sr_batch_loss_and_grad(sr_batch *b, const float *params_dev, double *losses_dev, double *total_dev,
                                 double *total_host, float *grad_dev) {
    if (!b || !params_dev || !grad_dev) return fail(SR_ERR_ARG, "NULL argument");
    if (sr_status st = batch_pts_check(b)) return st;
    Plan *pl = b->plan;
    pl->launches = run_eval(pl, params_dev, grad_dev, b->stream, nullptr);
    SR_CUDA(cudaGetLastError());
    if (losses_dev)
        SR_CUDA(cudaMemcpyAsync(losses_dev, pl->losses, sizeof(double) * pl->n_fields, cudaMemcpyDeviceToDevice, b->stream));
    if (total_dev) SR_CUDA(cudaMemcpyAsync(total_dev, pl->total, sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    if (total_host) {
        SR_CUDA(cudaMemcpyAsync(total_host, pl->total, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        SR_CUDA(cudaStreamSynchronize(b->stream));
        sr_status st = batch_check(b);
        if (st != SR_OK) return st;
        if ((st = pl->arena.check_guards()) != SR_OK) return st;
        for (sr_problem *p : b->probs)
            if ((st = p->arena.check_guards()) != SR_OK) return st;
        if (!std::isfinite(*total_host)) return fail(SR_ERR_NONFINITE, "the loss is not finite");
    }
    return SR_OK;
}

sr_status sr_batch_loss_and_grad_host(sr_batch *b, const float *params_host, double *total_host, float *grad_host) {
    if (!b || !params_host || !total_host || !grad_host) return fail(SR_ERR_ARG, "NULL argument");
    Plan *pl = b->plan;
    sr_status st;
    if ((st = ensure_opt_buffers(pl)) != SR_OK) return st;
    if (!pl->params_int && (st = pl->arena.alloc(&pl->params_int, pl->n_params)) != SR_OK) return st;
    if ((st = params_in(pl->params_int, params_host, pl->n_params, b->stream)) != SR_OK) return st;
    if ((st = sr_batch_loss_and_grad(b, pl->params_int, nullptr, nullptr, nullptr, pl->grad_int)) != SR_OK) return st;
    if ((st = results_out(grad_host, pl->grad_int, pl->n_params, total_host, pl->total, b->stream)) != SR_OK) return st;
    SR_CUDA(cudaStreamSynchronize(b->stream));
    if ((st = batch_check(b)) != SR_OK) return st;
    if (!std::isfinite(*total_host)) return fail(SR_ERR_NONFINITE, "the loss is not finite");
    return SR_OK;
}

// Queued form of the host-buffer evaluation: the same copies and launches on the batch's stream,
// no synchronisation; the inputs' checks wait for sr_batch_sync.
sr_status sr_batch_loss_and_grad_host_async(sr_batch *b, const float *params_host, double *total_host,
                                            float *grad_host) {
    if (!b || !params_host || !total_host || !grad_host) return fail(SR_ERR_ARG, "NULL argument");
    Plan *pl = b->plan;
    sr_status st;
    if ((st = ensure_opt_buffers(pl)) != SR_OK) return st;
    if (!pl->params_int && (st = pl->arena.alloc(&pl->params_int, pl->n_params)) != SR_OK) return st;
    if ((st = params_in(pl->params_int, params_host, pl->n_params, b->stream)) != SR_OK) return st;
    if ((st = sr_batch_loss_and_grad(b, pl->params_int, nullptr, nullptr, nullptr, pl->grad_int)) != SR_OK) return st;
    if ((st = results_out(grad_host, pl->grad_int, pl->n_params, total_host, pl->total, b->stream)) != SR_OK) return st;
    return SR_OK;
}

sr_status sr_batch_sync(sr_batch *b) {
    if (!b) return fail(SR_ERR_ARG, "NULL argument");
    SR_CUDA(cudaStreamSynchronize(b->stream));
    return batch_check(b);
}

sr_status sr_batch_step(sr_batch *b, float *params_dev, int n_steps, const sr_optim_cfg *cfg, double *last_total_host) {
    if (!b || !params_dev || !cfg || n_steps < 0) return fail(SR_ERR_ARG, "bad argument");
    if (sr_status st0 = batch_pts_check(b)) return st0;
    sr_status st = run_steps(b->plan, b->stream, params_dev, n_steps, cfg, nullptr, nullptr);
    if (st != SR_OK) return st;
    if (last_total_host) {
        SR_CUDA(cudaMemcpyAsync(last_total_host, b->plan->total, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        SR_CUDA(cudaStreamSynchronize(b->stream));
        if ((st = batch_check(b)) != SR_OK) return st;
    }
    return SR_OK;
}

// The table of the batched set-up: each member's buffers and shape, prefix offsets of the packed
// inputs, the kernel-spectra items, and a staging buffer for inputs that come from the host.
static sr_status batch_io_prepare(sr_batch *b) {
    if (b->bio_tab) return SR_OK;
    const int n = (int)b->probs.size();
    std::vector<BioEntry> tab(n);
    std::vector<long long> od(n + 1, 0), os(n + 1, 0), ok(n + 1, 0);
    std::vector<int2> items;
    for (int i = 0; i < n; ++i) {
        sr_problem *p = b->probs[i];
        const sr_problem_desc &d = p->desc;
        BioEntry &e = tab[i];
        e.d = p->d;
        e.w = p->w;
        e.s = p->s;
        e.kappa = p->kappa;
        e.flag = p->d_flag;
        e.E = d.n_epochs;
        e.N = d.data_n;
        e.K = d.psf_k;
        e.f = d.supersampling;
        e.Tk = p->Tk;
        e.tau_lo = p->tau_lo;
        od[i + 1] = od[i] + (long long)e.E * e.N * e.N;
        os[i + 1] = os[i] + (long long)e.E * e.K * e.K;
        ok[i + 1] = ok[i] + (long long)e.E * e.f * e.f * e.Tk * e.Tk;
        if (p->khat && !p->fft_big)
            for (int j = 0; j < e.E * ((e.f * e.f + 1) / 2); ++j) items.push_back(make_int2(i, j));
    }
    // items grouped by transform size: one launch per size with that size's block
    std::stable_sort(items.begin(), items.end(), [&](const int2 &a, const int2 &c) {
        return b->probs[a.x]->fft_L < b->probs[c.x]->fft_L;
    });
    for (size_t j = 0; j < items.size(); ++j) {
        const int L = b->probs[items[j].x]->fft_L;
        if (b->bio_ranges.empty() || b->bio_ranges.back()[0] != L) b->bio_ranges.push_back({L, (int)j, 0});
        ++b->bio_ranges.back()[2];
    }
    DevArena &A = b->bio_arena;
    sr_status st;
    if ((st = A.alloc(&b->bio_tab, (size_t)n)) != SR_OK) return st;
    if ((st = A.alloc(&b->bio_off_d, (size_t)n + 1)) != SR_OK) return st;
    if ((st = A.alloc(&b->bio_off_s, (size_t)n + 1)) != SR_OK) return st;
    if ((st = A.alloc(&b->bio_off_k, (size_t)n + 1)) != SR_OK) return st;
    if ((st = A.alloc(&b->bio_items, items.size())) != SR_OK) return st;
    if ((st = A.alloc(&b->bio_flags, (size_t)n)) != SR_OK) return st;
    const size_t stage_len[3] = {(size_t)od[n], (size_t)od[n], (size_t)os[n]};
    for (int k = 0; k < 3; ++k)
        if ((st = A.alloc(&b->bio_stage[k], stage_len[k])) != SR_OK) return st;
    SR_CUDA(cudaStreamCreateWithFlags(&b->bio_io, cudaStreamNonBlocking));
    for (int k = 0; k < 3; ++k) {
        SR_CUDA(cudaEventCreateWithFlags(&b->bio_free[k], cudaEventDisableTiming));
        SR_CUDA(cudaEventCreateWithFlags(&b->bio_copied[k], cudaEventDisableTiming));
        SR_CUDA(cudaEventRecord(b->bio_free[k], b->stream));
    }
    SR_CUDA(cudaMemcpy(b->bio_tab, tab.data(), sizeof(BioEntry) * n, cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemcpy(b->bio_off_d, od.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemcpy(b->bio_off_s, os.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemcpy(b->bio_off_k, ok.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    if (!items.empty())
        SR_CUDA(cudaMemcpy(b->bio_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    b->bio_total_d = od[n];
    b->bio_total_s = os[n];
    b->bio_total_k = ok[n];
    b->bio_vec_d = b->bio_vec_s = true;
    for (int i = 0; i <= n; ++i) {
        if (od[i] % 4) b->bio_vec_d = false;
        if (os[i] % 4) b->bio_vec_s = false;
    }
    return SR_OK;
}

static bool aligned16(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

// The packed input of kind k on the device: the caller's device array, or the kind's staging
// buffer after one copy on the internal stream (ordered as described at bio_stage).
static sr_status batch_io_source(sr_batch *b, int k, const float *src, long long count, int on_device,
                                 const float **out) {
    if (on_device) {
        *out = src;
        return SR_OK;
    }
    SR_CUDA(cudaStreamWaitEvent(b->bio_io, b->bio_free[k], 0));
    SR_CUDA(cudaMemcpyAsync(b->bio_stage[k], src, sizeof(float) * count, cudaMemcpyHostToDevice, b->bio_io));
    SR_CUDA(cudaEventRecord(b->bio_copied[k], b->bio_io));
    SR_CUDA(cudaStreamWaitEvent(b->stream, b->bio_copied[k], 0));
    *out = b->bio_stage[k];
    return SR_OK;
}

sr_status sr_batch_set_data(sr_batch *b, const float *d, int on_device) {
    if (!b || !d) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    const float *src;
    if ((st = batch_io_prepare(b)) != SR_OK) return st;
    if ((st = batch_io_source(b, 0, d, b->bio_total_d, on_device, &src)) != SR_OK) return st;
    launch_bio_data(b->bio_tab, b->bio_off_d, (int)b->probs.size(), src, b->bio_total_d,
                    b->bio_vec_d && aligned16(src), b->stream);
    SR_CUDA(cudaGetLastError());
    SR_CUDA(cudaEventRecord(b->bio_free[0], b->stream));
    b->bio_pending = true;
    return SR_OK;
}

sr_status sr_batch_set_noise(sr_batch *b, const float *sigma, int on_device) {
    if (!b || !sigma) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    const float *src;
    if ((st = batch_io_prepare(b)) != SR_OK) return st;
    if ((st = batch_io_source(b, 1, sigma, b->bio_total_d, on_device, &src)) != SR_OK) return st;
    launch_bio_noise(b->bio_tab, b->bio_off_d, (int)b->probs.size(), src, b->bio_total_d,
                     b->bio_vec_d && aligned16(src), b->stream);
    SR_CUDA(cudaGetLastError());
    SR_CUDA(cudaEventRecord(b->bio_free[1], b->stream));
    b->bio_pending = true;
    return SR_OK;
}

sr_status sr_batch_set_psfs(sr_batch *b, const float *s, int on_device) {
    if (!b || !s) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    const float *src;
    if ((st = batch_io_prepare(b)) != SR_OK) return st;
    if ((st = batch_io_source(b, 2, s, b->bio_total_s, on_device, &src)) != SR_OK) return st;
    launch_bio_psfs(b->bio_tab, b->bio_off_s, b->bio_off_k, (int)b->probs.size(), src, b->bio_total_s,
                    b->bio_total_k, b->bio_vec_s && aligned16(src), b->stream);
    SR_CUDA(cudaEventRecord(b->bio_free[2], b->stream));  // the staged PSFs are read by the copy kernel only
    for (const auto &r : b->bio_ranges)
        if ((st = launch_fft_kappa_pair_batch(b->plan->d_fields, b->bio_items + r[1], r[2], r[0], g_num_sms,
                                              b->stream)) != SR_OK)
            return st;
    for (sr_problem *p : b->probs)
        if (p->fft_big) {
            FieldDev fd;
            fill_field_common(fd, p);
            launch_big_kappa(fd, p->big_zb, p->big_zt, b->stream);
        }
    SR_CUDA(cudaGetLastError());
    b->bio_pending = true;
    return SR_OK;
}

sr_status sr_batch_lbfgsb(sr_batch *b, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                          sr_lbfgsb_info *info) {
    if (!b || !params_dev || !cfg) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    if ((st = batch_check(b)) != SR_OK) return st;
    sr_lbfgsb_cfg c;
    if ((st = lbfgsb_config(cfg, &c)) != SR_OK) return st;
    LbfgsbProblem P;
    P.n = (long long)b->plan->n_params;
    for (size_t i = 0; i < b->probs.size(); ++i)
        add_bounds(P, b->probs[i]->desc, b->probs[i]->F, (long long)b->plan->param_off[i]);
    P.eval = [b](const float *x, float *g, double *f) {
        return sr_batch_loss_and_grad(b, x, nullptr, nullptr, f, g);
    };
    return lbfgsb_run(P, params_dev, c, f_history, info, b->stream);
}

sr_status sr_batch_lbfgsb_fields(sr_batch *b, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                                 sr_lbfgsb_info *info, int *rounds) {
    if (!b || !params_dev || !cfg) return fail(SR_ERR_ARG, "NULL argument");
    sr_status st;
    if ((st = batch_check(b)) != SR_OK) return st;
    sr_lbfgsb_cfg c;
    if ((st = lbfgsb_config(cfg, &c)) != SR_OK) return st;
    LbfgsbFields P;
    P.n = (long long)b->plan->n_params;
    const int nf = (int)b->probs.size();
    for (int i = 0; i < nf; ++i) {
        const sr_problem *q = b->probs[i];
        LbfgsbProblem one;
        add_bounds(one, q->desc, q->F, (long long)b->plan->param_off[i]);
        P.off.push_back((long long)b->plan->param_off[i]);
        P.len.push_back((long long)param_count(q->desc));
        P.ranges.push_back(one.ranges);
        P.lo.push_back(one.lo);
    }
    P.eval = [b](const float *x, float *g, double *losses_dev) {
        double total = 0.0;
        return sr_batch_loss_and_grad(b, x, losses_dev, nullptr, &total, g);
    };
    return lbfgsb_fields_run(P, params_dev, c, f_history, info, rounds, b->stream);
}

sr_status sr_batch_reset_optimizer(sr_batch *b) {
    if (!b) return fail(SR_ERR_ARG, "NULL batch");
    Plan *pl = b->plan;
    sr_status st;
    if ((st = ensure_opt_buffers(pl)) != SR_OK) return st;
    SR_CUDA(cudaMemsetAsync(pl->opt_m, 0, sizeof(float) * pl->n_params, b->stream));
    SR_CUDA(cudaMemsetAsync(pl->opt_v, 0, sizeof(float) * pl->n_params, b->stream));
    SR_CUDA(cudaMemsetAsync(pl->d_t, 0, sizeof(long long), b->stream));
    return SR_OK;
}

int sr_batch_launches_per_eval(const sr_batch *b) { return b ? b->plan->launches : 0; }

int sr_batch_field_form(const sr_batch *b, int i) {
    if (!b || i < 0 || i >= b->plan->n_fields) return -1;
    return b->plan->h_fields[i].mode != 0 ? SR_CONV_FFT : SR_CONV_DIRECT;
}

sr_status sr_batch_profile(sr_batch *b, int enable) {
    if (!b) return fail(SR_ERR_ARG, "NULL batch");
    Plan *pl = b->plan;
    if (enable && pl->prof_ev.empty()) {
        pl->prof_ev.resize(4 * 512);
        for (cudaEvent_t &e : pl->prof_ev) SR_CUDA(cudaEventCreate(&e));
    }
    pl->profiling = enable != 0;
    pl->prof_count = 0;
    return SR_OK;
}

sr_status sr_batch_profile_read(sr_batch *b, int *n_evals, double *fwd_ms, double *adj_ms, double *fft_ms) {
    if (!b || !n_evals || !fwd_ms || !adj_ms || !fft_ms) return fail(SR_ERR_ARG, "NULL argument");
    Plan *pl = b->plan;
    *n_evals = 0;
    *fwd_ms = *adj_ms = *fft_ms = 0.0;
    if (pl->prof_ev.empty()) return SR_OK;
    SR_CUDA(cudaStreamSynchronize(b->stream));
    const int ring = (int)pl->prof_ev.size() / 4;
    const int n = std::min(pl->prof_count, ring);
    for (int i = 0; i < n; ++i) {
        float a = 0.f, c = 0.f, d = 0.f;
        SR_CUDA(cudaEventElapsedTime(&a, pl->prof_ev[4 * i], pl->prof_ev[4 * i + 1]));
        SR_CUDA(cudaEventElapsedTime(&c, pl->prof_ev[4 * i + 1], pl->prof_ev[4 * i + 2]));
        SR_CUDA(cudaEventElapsedTime(&d, pl->prof_ev[4 * i + 2], pl->prof_ev[4 * i + 3]));
        *fwd_ms += a;
        *adj_ms += c;
        *fft_ms += d;
    }
    *n_evals = n;
    return SR_OK;
}

}  // extern "C"
