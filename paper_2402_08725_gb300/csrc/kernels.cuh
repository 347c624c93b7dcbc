// Host-side launchers of the library's kernels (internal).
#pragma once

#include "common.cuh"

namespace sr {

// Outputs per thread of the register-blocked correlation (a compile-time width).
constexpr int kR = 16;
// Shared memory kept back from the opt-in limit for the static shared memory of the tile kernels
// (the work item, reduction slots and the staged point sources: under 2 KB).
constexpr int kTileStaticReserve = 2048;

// --- deconvolution (deconv.cu) ---
void launch_kappa_prep(const float *s, float *kappa, int E, int K, int f, int Tk, int tau_lo, cudaStream_t st);
int tile_smem_bytes(const TileItem &t, int Tk, bool fwd);
// phase groups of a tile: the most (a divisor of f^2) that fit one block and smem_limit bytes
int choose_tile_pg(int nph, TileItem t, int Tk, int smem_limit);
sr_status configure_tile_kernels(int smem_fwd, int smem_adj);
sr_status occupancy_tile_kernels(int smem_fwd, int smem_adj, int *blocks_fwd, int *blocks_adj);
void launch_fwd(const FieldDev *fields, const TileItem *items, int n_items, int *counter, const float *params,
                float *ebuf, double *chi_part, double *se_part, int grid, int smem, cudaStream_t st);
void launch_adj(const FieldDev *fields, const TileItem *items, int n_items, int *counter, const float *ebuf,
                float *gbuf, int grid, int smem, cudaStream_t st);
void launch_psgrad(const FieldDev *fields, const int4 *ps_items, int n, const float *params, const float *gbuf,
                   float *ps_da, float *ps_du, cudaStream_t st);
void launch_hgrad(const FieldDev *fields, const ChunkItem *chunks, int n_chunks, const float *gbuf, float *grad,
                  const float *params, cudaStream_t st);
// the moved extended channel's part of dL/d delta_i (fields with translate set; grid E_max x fields)
void launch_hshift_grad(const FieldDev *fields, int n_fields, int E_max, const float *params, const float *gbuf,
                        float *hs, cudaStream_t st);
// pts_fields / l1_pts / pts_g: the point-source prior's table and outputs (launch_pts_prior), or
// nullptr when no field of the table has the term
void launch_finalize(const FieldDev *fields, int n_fields, const double *chi_part, const double *se_part,
                     const double *l1_part, const float *ps_da, const float *ps_du, float *grad, double *losses,
                     double *total, cudaStream_t st, const FieldDev *pts_fields = nullptr,
                     const double *l1_pts = nullptr, const float *pts_g = nullptr, const float *hs = nullptr);

// --- frequency-domain form (fft_pair.cu): in-place transforms of real image pairs ---
bool fft_pair_size(int L);
int fft_pair_next(int need);  // smallest listed size >= need, 0 if none
int fft_pair_zn(int L);       // float2 elements of one pair array
int fft_pair_smem_bytes(int L, int M, int f, int GP);  // chunk kernel, GP epoch pairs per group
int fft_pair_field_smem(int L);                        // per-field and per-PSF kernels
bool fft_pair_variant(int L, int M, int GP);           // the chunk kernel is compiled for it
int fft_pair_gpmax(int L);                             // widest group of pairs (one source)
sr_status configure_fft_pair(int optin, int *chunk_limit, int *field_limit);
sr_status configure_fft_pair_field(int optin, int *field_limit);  // called by configure_fft_pair
// spectra of a problem's folded kernels (set_psfs): [E][f*f][L][L/2+2], the pad column zero
void launch_fft_kappa_pair(const FieldDev &fd, const float *kappa, float2 *khat, cudaStream_t st);
// the same for (entry, epoch * pairs + pair of phases) items of a table whose entries all have
// transform size L (each entry's kappa and fft_khat), a persistent grid over n_sms SMs
sr_status launch_fft_kappa_pair_batch(const FieldDev *fields, const int2 *items, int n_items, int L, int n_sms,
                                      cudaStream_t st);
void launch_fft_hhat_pair(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_pairs, int smem,
                          const float *params, float2 *hhat, cudaStream_t st);
// dL/dh of the transform fields: one block per (field, pair of phases) adds the work items'
// accumulators and transforms back; when those blocks are fewer than n_sms, the sums run first
// on one thread per spectral point into the first item's accumulator (max_points = the largest
// f^2 L (L/2 + 1) of the fields).  Returns the number of launches.
int launch_fft_hgrad_pair(const FieldDev *fields, const int *fft_fields, int n_fft_fields, int max_pairs, int smem,
                          float2 *acc, float *grad, int max_points, int n_sms, cudaStream_t st);
sr_status occupancy_fft_pair(int smem, int *blocks);
void launch_fft_chunks_pair(const FieldDev *fields, const int4 *items, int n_items, int *counter, const float *params,
                            const float2 *hhat, float2 *acc, double *chi_part, double *se_part, float *ps_da,
                            float *ps_du, int grid, int smem, cudaStream_t st);

// --- frequency-domain form through global memory (fft_big.cu): sizes beyond shared memory ---
// Per field and evaluation: zb and zt (the images and their transposes, E * pairs-of-phases * N * L
// complex each), fhat (the frames' spectra, E * f^2 * (L/2+1) * L) and acc (the adjoint spectra of
// each pair of frames, ceil(E/2) * f^2 * (L/2+1) * L).
struct BigBuffers {
    float2 *zb, *zt, *fhat, *acc;
};
int fft_big_next(int need);                 // smallest size >= need of the global-memory list, 0 if none
int fft_big_window_smem(int Tk, int f);     // shared memory of the source-window adjoint kernel
sr_status configure_fft_big(int optin);
// kernel spectra [E][f^2][L/2+1][L] (transposed half spectra) at fd.fft_khat, with scratch zb, zt of
// E * pairs * Tk * L complex each
int launch_big_kappa(const FieldDev &fd, float2 *zb, float2 *zt, cudaStream_t st);
// the model, residual, chi^2 / sum e partial sums (n_tiles = N slots per epoch), the adjoint spectra
// and the source windows' adjoint images (gbuf); returns the number of launches
int launch_big_eval(const FieldDev &fd, const float *params, const BigBuffers &bb, float *ebuf, float *gbuf,
                    double *chi_part, double *se_part, cudaStream_t st);
// dL/dh of the field (after the starlet kernels, whose gradient it adds)
int launch_big_hgrad(const FieldDev &fd, const BigBuffers &bb, float *grad, cudaStream_t st);

// --- batched input set-up (batch_io.cu) ---
// One entry per problem of a batch: its device buffers and shape, for the packed inputs of
// sr_batch_set_data / _noise / _psfs (each problem's block at its prefix offset).
struct BioEntry {
    float *d, *w, *s, *kappa;
    int *flag;
    int E, N, K, f, Tk, tau_lo;
};
// vec: every offset and the total are multiples of 4 and src is 16-byte aligned (float4 moves)
void launch_bio_data(const BioEntry *tab, const long long *off, int n, const float *src, long long total, bool vec,
                     cudaStream_t st);
void launch_bio_flags(const BioEntry *tab, int n, int *out, cudaStream_t st);
void launch_bio_noise(const BioEntry *tab, const long long *off, int n, const float *src, long long total, bool vec,
                      cudaStream_t st);
void launch_bio_psfs(const BioEntry *tab, const long long *off_s, const long long *off_k, int n, const float *src,
                     long long total_s, long long total_k, bool vec, cudaStream_t st);
// n floats src -> dst and (when tdst is not null) one double tsrc -> tdst in one kernel; either side
// may be the mapped address of page-locked host memory
void launch_host_copy(const float *src, float *dst, long long n, const double *tsrc, double *tdst, cudaStream_t st);

// --- starlet prior (starlet.cu) ---
// Forward levels then adjoint levels for every field of the table (n_fields of them, grids at
// most Fmax wide); writes the per-(level, chunk) prior partial sums and leaves T0 = dP/dh in
// plane J of each field's starlet scratch.  starlet_field_form(F, J) says how a field runs: 0 as
// row bands, 1 as comb tiles, 3 as comb bands (2: no form, which no valid shape has); forms has
// bit 1 << form set for every form of the table's fields, and kStarletMapBit when some field has
// a per-coefficient weight map (chunks and n_chunks are not used).  Returns the number of launches
// issued.
constexpr int kStarletMapBit = 16;
// bits of forms that shorten the comb-band blocks to 4 or 8 rows (starlet_comb_rows_bits)
constexpr int kStarletRows4 = 32, kStarletRows8 = 64;
int starlet_field_form(int F, int J);
int starlet_comb_rows_of(int forms);
int starlet_comb_rows_bits(const int *F, const int *J, int n, int n_sms);
// forms of a table holding one field (with or without a weight map)
int starlet_forms_single(int F, int J, bool map);
int launch_starlet(const FieldDev *fields, int n_fields, int Fmax, int forms, const ChunkItem *chunks,
                   int n_chunks, int Jmax, const float *params, double *l1_part, cudaStream_t st);

// --- point-source prior and lambda_pts estimate (pts.cu) ---
// Shadow entries sh[0..n_sh) (each a copy of its field's entry with c_0 = the mean point-source
// image at param_off in pbar, lambda 1, weights lambda_pts W_j, its own starlet scratch, l1 slots
// in l1_pts and source slots ps_slot in abar / pts_g): value partial sums in l1_pts and per source
// (sum G r, d/dc_x, d/dc_y) in pts_g.  Returns the number of launches.
int launch_pts_prior(const FieldDev *sh, const FieldDev *fields, int n_sh, int Fmax, int Mmax, int starlet_forms,
                     const ChunkItem *chunks, int n_chunks, int Jmax, const float *params, float *abar, float *pbar,
                     double *l1_pts, float *pts_g, cudaStream_t st);
// The App. C ratio for one field (fd.param_off into params); synchronises st.
sr_status pts_estimate(const FieldDev &fd, const float *params, const float *Wd, float lambda, double *out_host,
                       cudaStream_t st);

// --- PSF reconstruction (psf.cu) ---
struct PsfBuffers {
    float *ebuf;        // [S][N][N]
    double *star_part;  // [S][n_dchunks][4]: chi2, da, dcx, dcy
    double *ab_part;    // [n_chunks][2]: dalpha, dbeta partials
    int n_dchunks;      // data-grid chunks per star
};
int launch_psf_eval(const FieldDev *fields, const FieldDev &host_field, const ChunkItem *chunks, int n_chunks,
                    const float *params, float *grad, const PsfBuffers &pb, double *l1_part, double *losses,
                    double *total, cudaStream_t st);

// The narrow PSF s = Moffat(alpha, beta) + b of the parameters, into fields[0].psf_s.
void launch_psf_model(const FieldDev *fields, int F, const float *params, cudaStream_t st);

// --- plain per-epoch form (plain.cu) ---
struct PlainBuffers {
    float *fimg;   // [F][F] rasterised fine image of the current epoch
    float *conv;   // [F][F] S_i f_i on the fine grid
    float *ey;     // [F][F] D^T e
    float *gsum;   // [F][F] running sum over epochs of S_i^T D^T e_i
    float *gi;     // [F][F] S_i^T D^T e_i of the current epoch
};
int launch_plain_eval(const FieldDev *fields, const FieldDev &hf, const float *s_raw, const ChunkItem *chunks,
                      int n_chunks, const float *params, float *grad, const PlainBuffers &pb, float *ebuf,
                      double *chi_part, double *se_part, float *ps_da, float *ps_du, const int4 *ps_items,
                      double *l1_part, double *losses, double *total, cudaStream_t st);
sr_status configure_plain_kernels(int K);

// --- optimiser (optim.cu) ---
struct OptimArgs {
    int kind;
    float beta1, beta2, eps;
    float lr[SR_MAX_GROUPS];
    float lo[SR_MAX_GROUPS];
};
void launch_opt_step(long long n, float *params, const float *grad, float *m, float *v, const uint8_t *group,
                     const OptimArgs &a, long long *t_dev, float *bc_dev, cudaStream_t st);

// --- input preparation (prep.cu) ---
void launch_inv_var(const float *sigma, float *w, long long n, int *bad_flag, cudaStream_t st);
void launch_check_finite(const float *x, long long n, int *bad_flag, cudaStream_t st);
// *loss = NaN if *flag is set (an input the weights could not be formed from)
void launch_flag_to_nan(const int *flag, double *loss, cudaStream_t st);

}  // namespace sr
