/*
 * starred.h — C ABI of the GB300 (sm_103a) STARRED loss-and-gradient library.
 *
 * The library evaluates, on one GPU, the regularised loss and its gradient of
 * STARRED (Millon et al., arXiv 2402.08725):
 *
 *  - joint multi-epoch two-channel deconvolution (sec. 2.2, Eq. 9-11 with
 *    lambda_pts = 0): per epoch i the fine image f_i = h + sum_k a_ki r_k is
 *    convolved with the epoch's narrow PSF s_i (operator S_i), block-summed to
 *    the data grid (operator D, the subsampling arrow of Eq. 1), compared with
 *    the data under diagonal inverse-variance weights (Eq. 10), and the
 *    starlet prior lambda ||W o Phi^T h||_1 (Eq. 6) is added;
 *  - PSF reconstruction (sec. 2.1, Eq. 2-4 and Eq. 7): narrow PSF
 *    s = Moffat(alpha, beta) + b, star k modelled as D(a_k (s * r_k)) with r_k
 *    the 2-pixel-FWHM Gaussian shifted to the star centre (Eq. 3), plus the
 *    starlet prior on b;
 *  - the gradient-based optimiser step the paper uses (sec. 2.4: AdaBelief;
 *    Adam is also offered), with projection a >= 0.
 *
 * Conventions (fixed readings of points the paper leaves open):
 *   Fine grid F = f*N (f = supersampling).  Arrays are row-major [row][col];
 *   2-vectors are (x, y) with x along columns.  Fine pixel u has data
 *   coordinate (u + 0.5)/f - 0.5; a point source at offset c (data pixels from
 *   the stamp centre (N-1)/2) sits at fine coordinate (F-1)/2 + f*c.
 *   Narrow PSFs are K x K with origin (K/2, K/2) (integer division); S is a
 *   true (flipped-kernel) linear convolution with zero padding and F x F output.
 *   D is a flux-conserving block sum of f x f fine pixels.
 *   The Gaussian r has FWHM 2 fine pixels, unit flux, point-sampled (Eq. 1).
 *   The per-epoch background Gamma_i (Eq. 9) adds f^2 * Gamma_i to every data
 *   pixel after D.  The per-epoch shift delta_i moves the point sources only.
 *   Starlet: isotropic undecimated B3-spline (1-4-6-4-1)/16 with holes 2^j,
 *   whole-sample mirror borders; J counts all planes (J-1 detail planes are
 *   penalised with weight W[j], the coarse plane is not); needs
 *   2 * 2^(J-2) <= F - 1.
 *   Noise: weights w = 1/sigma^2 (C diagonal, Eq. 4 and Eq. 10); sigma = +inf
 *   masks a pixel.
 *
 * Packed parameter vector (float32, device memory, owned by the caller):
 *   DECONV: [ h F*F | a E*M | c M*2 | delta E*2 | Gamma E ]
 *   PSF:    [ b F*F | alpha, beta | a S | c S*2 ]          (S = number of stars)
 *
 * Precision: FP32 arithmetic; the chi^2 and prior sums are accumulated in
 * FP64.  The loss is returned as a double.
 *
 * Ownership and streams: set_* calls copy the caller's arrays into device
 * buffers the library allocates at create time and frees at destroy; the
 * caller keeps its arrays.  Parameter and gradient pointers are caller-owned
 * device pointers that must stay valid until the call's work has finished on
 * the problem's stream.  All work is ordered on the stream given at create
 * (a cudaStream_t, NULL for the legacy default stream).  Calls that return a
 * value to a host pointer synchronise that stream; calls that write only to
 * device pointers do not.
 *
 * Errors: every call returns an sr_status; nothing is thrown across the ABI.
 * sr_last_error() gives a message for the calling thread's last failure.
 * Calls that need data not yet set return SR_ERR_STATE.  Non-finite inputs
 * (NaN data, NaN or non-positive sigma, non-finite PSF values) are rejected
 * with SR_ERR_NONFINITE by the first call after them that returns a host value.
 * Debugging aid: with the environment variable SR_GUARD=1 set when buffers are
 * allocated, every device buffer of the library carries a guard tail, and the
 * calls that return a host value fail with SR_ERR_STATE if a tail was written.  A problem is not thread-safe: use one per thread or
 * serialise calls.
 */
#ifndef STARRED_H
#define STARRED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SR_OK = 0,
    SR_ERR_ARG = 1,         /* null pointer, out-of-range argument */
    SR_ERR_SHAPE = 2,       /* inconsistent or unsupported sizes */
    SR_ERR_STATE = 3,       /* required data not set, or wrong problem kind */
    SR_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
    SR_ERR_OOM = 5,         /* device or host allocation failed */
    SR_ERR_NONFINITE = 6,   /* NaN/Inf input or non-finite loss */
    SR_ERR_TIMEOUT = 7,     /* a bounded device wait gave up */
    SR_ERR_UNSUPPORTED = 8  /* valid request that the library does not support */
} sr_status;

typedef enum { SR_DECONV = 0, SR_PSF = 1 } sr_kind;

/* How S (and D) are evaluated.  DIRECT is the fused D-folded direct form
 * (shared-memory tiles).  FFT evaluates the same folded form with circular
 * transforms whose size leaves the N x N output free of wrap-around (exact up
 * to rounding); it needs the transform buffers of one epoch to fit in shared
 * memory (SR_ERR_UNSUPPORTED at create otherwise).  AUTO uses FFT where it
 * fits, else DIRECT.  PLAIN is the literal per-epoch form (fine-grid
 * convolution, then D, residual, D^T, correlation, each a separate launch per
 * epoch), kept as the measured baseline. */
typedef enum { SR_CONV_AUTO = 0, SR_CONV_DIRECT = 1, SR_CONV_PLAIN = 2, SR_CONV_FFT = 3 } sr_conv_mode;

typedef struct {
    int kind;            /* sr_kind */
    int n_epochs;        /* DECONV: E epochs; PSF: S star cutouts */
    int data_n;          /* N: data stamps are N x N (1 <= N <= 4096) */
    int supersampling;   /* f >= 1: fine grid F = f*N */
    int psf_k;           /* DECONV: narrow PSF size K (1 <= K <= 511); PSF: ignored */
    int n_sources;       /* DECONV: point sources M (0 <= M <= 64); PSF: ignored */
    int n_scales;        /* J >= 2 starlet planes including the coarse one (<= 8) */
    double lambda;       /* prior strength lambda >= 0 (noise-sigma units, Eq. 6) */
    int conv_mode;       /* sr_conv_mode */
} sr_problem_desc;

/* Parameter groups of the packed vector, in order.
 * DECONV: 0 h, 1 a, 2 c, 3 delta, 4 Gamma.  PSF: 0 b, 1 (alpha, beta), 2 a, 3 c. */
#define SR_MAX_GROUPS 8
typedef struct {
    int n_groups;
    size_t offset[SR_MAX_GROUPS];
    size_t count[SR_MAX_GROUPS];
    size_t total;
} sr_layout;

typedef enum { SR_ADABELIEF = 0, SR_ADAM = 1 } sr_optim_kind;

/* Optimiser settings (sec. 2.4).  AdaBelief is the published update of
 * Zhuang et al. (2020): m = b1 m + (1-b1) g; s = b2 s + (1-b2)(g-m)^2 + eps;
 * theta -= lr * mhat / (sqrt(shat) + eps) with bias corrections.  Adam uses
 * g^2 in place of (g-m)^2 and no eps inside s.  lr is per parameter group
 * (sr_layout order).  After the update, a (both kinds) is projected onto
 * a >= 0, and for PSF problems alpha >= 1e-3 and beta >= 1.001. */
typedef struct {
    int kind;                   /* sr_optim_kind */
    float beta1, beta2, eps;
    float lr[SR_MAX_GROUPS];
} sr_optim_cfg;

typedef struct sr_problem sr_problem;
typedef struct sr_batch sr_batch;

/* Thread-local message describing the calling thread's last error ("" if none). */
const char *sr_last_error(void);

/* Library version and the device compute capability it was built for (103). */
int sr_version(void);
int sr_build_arch(void);

/* Create a problem on the current CUDA device.  Validates desc (SR_ERR_SHAPE
 * for sizes the method does not define, e.g. a starlet wider than the grid),
 * allocates all device buffers the problem needs, and binds `cuda_stream`.
 * On failure *out is NULL and nothing is leaked. */
sr_status sr_create_problem(const sr_problem_desc *desc, void *cuda_stream, sr_problem **out);

/* Free everything the problem owns.  NULL is accepted.  Synchronises the stream. */
sr_status sr_destroy(sr_problem *p);

/* Data d_i (Eq. 8 / Eq. 10; for PSF problems the star cutouts t_k of Eq. 3):
 * float32 [E][N][N], host (on_device = 0) or device (1) pointer.  Must be
 * finite.  The set_* calls do not synchronise: the copy is ordered on the
 * problem's stream (from page-locked host memory it is asynchronous, so keep
 * the array unchanged until the next synchronising call), and the finiteness
 * check runs on the device; a bad input makes the next call that returns a
 * host value fail with SR_ERR_NONFINITE. */
sr_status sr_set_data(sr_problem *p, const float *d, int on_device);

/* Noise standard deviation sigma (diagonal C of Eq. 4 / Eq. 10):
 * float32 [E][N][N]; each value > 0, or +inf to mask the pixel. */
sr_status sr_set_noise(sr_problem *p, const float *sigma, int on_device);

/* Narrow PSFs s_i of the epochs (sec. 2.2): float32 [E][K][K], origin
 * (K/2, K/2).  DECONV only (SR_ERR_STATE for PSF problems).  The library folds
 * D into each kernel here (kappa_i(t) = sum of s_i over an f x f block), so the
 * per-evaluation work uses the folded form. */
sr_status sr_set_psfs(sr_problem *p, const float *s, int on_device);

/* Prior weights W, one per detail scale (Eq. 6; sec. 2.3 gives their meaning):
 * float32 [J-1], host pointer, each finite and >= 0 (checked at once,
 * SR_ERR_NONFINITE otherwise); the array may be reused when the call returns. */
sr_status sr_set_weights(sr_problem *p, const float *W);

/* Prior weights per coefficient instead of per scale (sec. 2.3 and App. B propagate the noise to
 * a map W_j(u) per scale; sr_noise_weights returns it): the prior becomes
 *   lambda sum_j sum_u W_j(u) |w_j(u)|
 * (and lambda_pts times the same map for the point-source prior).  Wmap: float32 [J-1][F][F],
 * host (on_device = 0) or device pointer, each entry finite and >= 0 (SR_ERR_NONFINITE otherwise);
 * copied, so the array may be reused when the call returns; NULL clears the map and the per-scale
 * weights of sr_set_weights apply again.  Counts as setting the weights.  Later maps take effect at
 * the next evaluation (captured optimiser steps included); setting the first map or clearing it
 * drops the problem's plan and optimiser state, and a batch created before that returns
 * SR_ERR_STATE until it is re-created.  sr_estimate_lambda_pts returns SR_ERR_UNSUPPORTED while a
 * map is set.  Synchronises the problem's stream; allocates (J-1) F^2 floats on the first map. */
sr_status sr_set_weight_map(sr_problem *p, const float *Wmap, int on_device);

/* Point-source prior, the third term of Eq. 11 (sec. 2.2):
 *   lambda_pts || W o Phi^T sum_k <a_k> r_k ||_1,
 * <a_k> = (1/E) sum_i a_ki the mean amplitude of source k over the epochs, r_k the unit Gaussian
 * of Eq. 1 at its centre c_k (no per-epoch shift), W the prior weights of sr_set_weights.  DECONV
 * only (SR_ERR_STATE otherwise); lambda_pts finite and >= 0 (SR_ERR_ARG).  The default is 0 and
 * the term is then not evaluated.  The first non-zero value allocates the term's buffers and adds
 * it to the problem's evaluation (an existing optimiser state carries over); later values, zero
 * included, only change its weights, also inside captured optimiser steps.  A batch created
 * before a member's first non-zero value returns SR_ERR_STATE until it is re-created.  The plain
 * form (SR_CONV_PLAIN) evaluates lambda_pts = 0 only (SR_ERR_UNSUPPORTED at its next evaluation). */
sr_status sr_set_lambda_pts(sr_problem *p, double lambda_pts);

/* Move the extended channel with each epoch's shift (sec. 5, the frame shifts of the data set):
 * when enabled, epoch i sees h translated by f * delta_i fine pixels, delta_i the epoch's shift in
 * the packed parameters, by bilinear interpolation with zero outside the fine grid (the paper does
 * not fix the interpolant; this is the reading), and the gradient gains the shift derivative of
 * that term.  Off (0) by default: the paper's Eq. 8 applies the shift to the point sources only.
 * DECONV only (SR_ERR_STATE otherwise); SR_ERR_UNSUPPORTED with conv_mode FFT or PLAIN; under AUTO
 * the problem is evaluated in the direct form while enabled.  A change drops the problem's plan
 * and its optimiser state (synchronises the stream).  A batch created before a member's change
 * returns SR_ERR_STATE until it is re-created. */
sr_status sr_set_translate_h(sr_problem *p, int enable);

/* Rotated frames (sec. 5 names rotations between frames; no equation in the paper, so this is the
 * reading): epoch i's frame is the reference frame turned by theta[i] radians about the grid
 * centre u0 = (F - 1)/2 and, when sr_set_translate_h is on, shifted by f * delta_i.  Fine pixel u of
 * the epoch sees the extended channel at q = u0 + R^T (u - u0 - s), R = [[cos, -sin], [sin, cos]]
 * on (x, y), bilinear with zero outside the grid, and point source k sits at u0 + f (R c_k +
 * delta_i); the angles are fixed inputs (no gradient).  theta: host array of n_epochs finite
 * doubles (copied; SR_ERR_NONFINITE otherwise), or NULL to turn the rotations off.  DECONV only
 * (SR_ERR_STATE otherwise); SR_ERR_UNSUPPORTED with conv_mode FFT or PLAIN; under AUTO the problem
 * is evaluated in the direct form while they are on.  New angles take effect at the next evaluation
 * (captured optimiser steps included); turning them on or off drops the problem's plan and its
 * optimiser state, and a batch created before that returns SR_ERR_STATE until it is re-created.
 * The point-source prior and the App. C estimate stay in the reference frame.  Synchronises the
 * problem's stream; allocates 2 n_epochs floats on the first call. */
sr_status sr_set_rotations(sr_problem *p, const double *theta);

/* lambda_pts from a model, by the ratio of App. C:
 *   lambda (|| W o Phi^T fbar ||_1 - || W o Phi^T h ||_1) / sum_k <a_k> || W o Phi^T r_k ||_1,
 * fbar = (1/E) sum_i (h + sum_k a_ki r_k(c_k + delta_i)) the mean of the epochs' fine images,
 * h and r_k (unit Gaussian at c_k) as above, lambda the problem's.  (The printed ratio also
 * multiplies the second norm by lambda; it is read without that factor, which would leave the
 * difference without a consistent unit.)  0 when the denominator is 0.  The paper starts from
 * 0.5 lambda and refines the value from each best fit until it settles.  params_dev: the packed
 * DECONV vector (device); *lambda_pts receives the value; synchronises the stream; allocates and
 * frees a workspace of 2 (M + 2) F^2 floats.  SR_ERR_STATE without weights or for PSF problems. */
sr_status sr_estimate_lambda_pts(sr_problem *p, const float *params_dev, double *lambda_pts);

/* Number of float32 values in the packed parameter vector, and its layout. */
size_t sr_param_count(const sr_problem *p);
sr_status sr_param_layout(const sr_problem *p, sr_layout *out);

/* Loss L (Eq. 11 for DECONV, Eq. 7 for PSF) at params (device pointer).
 * Writes *loss_host; synchronises the stream. */
sr_status sr_loss(sr_problem *p, const float *params_dev, double *loss_host);

/* Loss and gradient dL/dparams (same packed layout) at params.  grad_dev is a
 * device pointer with sr_param_count floats; it is fully overwritten.  The loss
 * goes to loss_dev (device double, no synchronisation) and/or loss_host
 * (synchronises); either may be NULL.  Returns SR_ERR_NONFINITE if a host loss
 * was requested and it is not finite. */
sr_status sr_loss_and_grad(sr_problem *p, const float *params_dev, double *loss_host, double *loss_dev,
                           float *grad_dev);

/* End-to-end variant with HOST buffers: copies params_host (sr_param_count
 * floats) to the device, evaluates, and copies the gradient back to grad_host
 * and the loss to *loss_host.  Synchronises.  For best throughput the host
 * buffers should be page-locked: from and to page-locked memory (as for the
 * host arrays of sr_set_data / _noise / _psfs) the library moves the values
 * with kernels through the memory's mapped address rather than the copy
 * engines, so that its transfers never wait in an engine's queue ahead of
 * other streams' copies. */
sr_status sr_loss_and_grad_host(sr_problem *p, const float *params_host, double *loss_host, float *grad_host);
/* The same, queued without waiting: returns once the copies and the evaluation
 * are queued on the problem's stream.  params_host must stay unchanged and
 * grad_host / *loss_host untouched until sr_sync (or any synchronisation of
 * the stream) returns; the loss is not checked for finiteness (the caller
 * reads it).  With pageable buffers the copies may block the host. */
sr_status sr_loss_and_grad_host_async(sr_problem *p, const float *params_host, double *loss_host, float *grad_host);
/* Waits for the problem's stream and reports the input checks of the set-up
 * calls since the last check (SR_ERR_NONFINITE). */
sr_status sr_sync(sr_problem *p);

/* Optimiser: run n_steps of {loss_and_grad; update} on params_dev in place.
 * The moment buffers and step counter live in the problem (sr_reset_optimizer
 * clears them; sr_get_state/sr_set_state save and restore them).  The steps
 * are captured once as a CUDA graph and replayed.  losses_dev (nullable,
 * device, n_steps doubles) receives the loss before each update;
 * last_loss_host (nullable) receives the last one and synchronises. */
sr_status sr_step(sr_problem *p, float *params_dev, int n_steps, const sr_optim_cfg *cfg, double *losses_dev,
                  double *last_loss_host);
sr_status sr_reset_optimizer(sr_problem *p);
/* Optimiser state as plain buffers: m and v (device, sr_param_count floats
 * each) and the 1-based count of updates done.  Restoring a saved state makes
 * the following steps bitwise identical to an uninterrupted run. */
sr_status sr_get_state(sr_problem *p, float *m_dev, float *v_dev, int64_t *t);
sr_status sr_set_state(sr_problem *p, const float *m_dev, const float *v_dev, int64_t t);

/* Batch of independent DECONV problems (fields of uneven sizes, epoch counts
 * and starlet depths) evaluated together: every kernel of the evaluation runs
 * once for all fields (persistent launches over one work list sorted by cost).
 * The problems must be fully set (data, noise, PSFs, weights) and must outlive
 * the batch; later set_* calls on them are seen by the batch.  The batch's
 * parameter vector is the concatenation of the fields' packed vectors;
 * sr_batch_param_offset gives field i's offset.  1 <= n <= 65535 (fields index a
 * grid dimension); otherwise SR_ERR_ARG. */
sr_status sr_batch_create(sr_problem *const *problems, int n, void *cuda_stream, sr_batch **out);

/* The inputs of every member at once: the arrays of the members' sr_set_data / sr_set_noise /
 * sr_set_psfs calls concatenated in batch order (float32, host or device as on_device says;
 * page-locked host memory makes the single copy asynchronous).  The same effect as those calls on
 * each member, with one host-to-device copy and a few launches for the whole batch (the PSFs'
 * folding and, for members of the transform form, their kernel spectra included), ordered on the
 * batch's stream; the members' own streams must have no set-up or evaluation of these members in
 * flight.  From host memory each kind is staged by a copy on an internal stream that overlaps
 * the set-up of the other kinds (calling sr_batch_set_psfs first lets its folding and spectra run
 * under the data and noise copies); the host array must stay valid until the batch's stream has
 * passed the call.  Checks and errors as the per-member calls (reported by the next call that
 * returns a host value).  The first call allocates a table of the members and one staging buffer
 * per kind (the packed data, noise and PSF sizes). */
sr_status sr_batch_set_data(sr_batch *b, const float *d, int on_device);
sr_status sr_batch_set_noise(sr_batch *b, const float *sigma, int on_device);
sr_status sr_batch_set_psfs(sr_batch *b, const float *s, int on_device);
sr_status sr_batch_destroy(sr_batch *b);
size_t sr_batch_param_count(const sr_batch *b);
sr_status sr_batch_param_offset(const sr_batch *b, int i, size_t *offset);
/* losses_dev (nullable, device, n doubles): loss of each field.  total_dev
 * (nullable, device double) and total_host (nullable, synchronises): sum over
 * fields.  grad_dev: device, sr_batch_param_count floats, fully overwritten. */
sr_status sr_batch_loss_and_grad(sr_batch *b, const float *params_dev, double *losses_dev, double *total_dev,
                                 double *total_host, float *grad_dev);
/* End-to-end variant with HOST buffers (see sr_loss_and_grad_host). */
sr_status sr_batch_loss_and_grad_host(sr_batch *b, const float *params_host, double *total_host, float *grad_host);
/* The same evaluation queued without waiting: the parameters' copy in, the evaluation and the
 * copies of the gradient and the total out are ordered on the batch's stream, and the call
 * returns once they are queued.  Successive calls with batched set-up between them pipeline:
 * the next step's input copies (sr_batch_set_* from host memory, staged on the internal stream)
 * run while this step computes.  With page-locked host buffers nothing blocks the host;
 * params_host must stay unchanged and grad_host / total_host untouched until sr_batch_sync (or
 * any synchronisation of the batch's stream) returns.  Input checks (non-finite values, sigma
 * <= 0) are gathered over every queued step and reported by sr_batch_sync; the totals are not
 * checked for finiteness (the caller reads them). */
sr_status sr_batch_loss_and_grad_host_async(sr_batch *b, const float *params_host, double *total_host,
                                            float *grad_host);
/* Waits for everything queued on the batch's stream and reports the input checks of the batched
 * set-up calls since the last check (SR_ERR_NONFINITE names the first field concerned). */
sr_status sr_batch_sync(sr_batch *b);
/* n_steps optimiser updates of all fields at once (same cfg for every field),
 * captured as one CUDA graph and replayed. */
sr_status sr_batch_step(sr_batch *b, float *params_dev, int n_steps, const sr_optim_cfg *cfg,
                        double *last_total_host);
sr_status sr_batch_reset_optimizer(sr_batch *b);

/* Which form evaluates field i of the batch: SR_CONV_DIRECT or SR_CONV_FFT
 * (AUTO fields are resolved by the autotuner when the batch is created: both
 * forms are timed on the field's shape and the faster one is kept; the
 * choices are cached per shape in memory, and in the JSON file named by the
 * environment variable SR_AUTOTUNE_CACHE when it is set).  -1 for a bad
 * argument. */
int sr_batch_field_form(const sr_batch *b, int i);

/* Schedule of the transform form (the paper has no counterpart: it decides how
 * the epochs of sec. 2.4's joint evaluation are spread over the GPU, not what is
 * computed).  The per-epoch kernel takes work items of epochs_per_item
 * consecutive epochs of one field (each with its own accumulator of adjoint
 * spectra) and transforms pairs_per_group = 1 epoch pair at a time, or (0) the
 * widest group of pairs compiled for the field's transform size.  By default a
 * batch takes as many epochs per item as keep at least two items per SM (even,
 * 2 .. 16).  sr_batch_set_schedule rebuilds the batch's plan with the given
 * schedule (epochs_per_item 0 or even in 2 .. 16; pairs_per_group 0 or 1;
 * SR_ERR_ARG otherwise); it synchronises the batch's stream and drops its
 * captured optimiser graph.  Results differ between schedules only by the
 * order of FP32 sums of the adjoint spectra.  sr_batch_get_schedule gives the
 * schedule in use (epochs per item, pair cap).  sr_batch_tune_schedule times
 * one warm-up and three evaluations of each candidate (2, 4, 8, 16 epochs per
 * item, each with and without the pair cap) on zero parameters, keeps the
 * fastest and caches it by a digest of the fields' shapes and forms (in memory,
 * and in the SR_AUTOTUNE_CACHE file when set); a cached schedule is applied
 * without timing (*ms_per_eval = -1).  Output pointers may be NULL. */
sr_status sr_batch_set_schedule(sr_batch *b, int epochs_per_item, int pairs_per_group);
sr_status sr_batch_get_schedule(const sr_batch *b, int *epochs_per_item, int *pairs_per_group);
sr_status sr_batch_tune_schedule(sr_batch *b, int *epochs_per_item, int *pairs_per_group, float *ms_per_eval);

/* Launch statistics of the last evaluation on this problem/batch: number of
 * kernel launches one loss_and_grad issues. */
int sr_launches_per_eval(const sr_problem *p);
int sr_batch_launches_per_eval(const sr_batch *b);

/* Kernel timing: while enabled, every evaluation of the batch records CUDA
 * events on the batch's stream around its hot kernels — the forward and the
 * adjoint tile kernels of the fields in the direct form, and the transform
 * kernels (h spectra and the per-epoch kernel) of the fields in the FFT form
 * (a ring of the last 512 evaluations); sr_batch_step runs without graph
 * capture meanwhile.  enable = 1 also clears the record. */
sr_status sr_batch_profile(sr_batch *b, int enable);
/* Evaluations recorded and the summed durations in milliseconds of the
 * forward tile kernel, the adjoint tile kernel and the transform kernels.
 * Synchronises the batch's stream. */
sr_status sr_batch_profile_read(sr_batch *b, int *n_evals, double *fwd_ms, double *adj_ms, double *fft_ms);

/* Diagnostic, not from the paper: measured FP32 fused-multiply-add throughput of the current
 * CUDA device in TFLOP/s (a register-resident FMA kernel on the legacy default stream, timed
 * with events after a warm-up; synchronises the device's default stream).  It is the
 * denominator of the direct form's roofline, whose tile kernels are bound by FP32 FMA issue.
 * *tflops receives the figure; SR_ERR_CUDA if a CUDA call fails. */
sr_status sr_measure_fp32_peak(double *tflops);

/* The reconstructed narrow PSF of a PSF fit (sec. 2.1, Eq. 2): s = Moffat(alpha, beta) + b on the
 * F x F fine grid, the Moffat part centred on fine pixel (F/2, F/2) with unit analytic flux.
 * params_dev: the packed PSF vector (device); s_dev: F*F floats (device), written on the
 * problem's stream (no synchronisation).  SR_ERR_STATE for a deconvolution problem. */
sr_status sr_psf_model(sr_problem *p, const float *params_dev, float *s_dev);

/* L-BFGS-B, the paper's second optimiser (sec. 2.4; the algorithm of Byrd, Lu, Nocedal & Zhu 1995:
 * compact limited-memory matrix, generalised Cauchy point, subspace minimisation, strong-Wolfe
 * line search by bracketing and bisection with c1 = 1e-3, c2 = 0.9, steps in (0, 1]).  Bounds:
 * the same lower bounds as the sr_step projection (amplitudes >= 0; for a PSF fit also
 * alpha >= 1e-3 and beta >= 1.001), no others. */
typedef struct {
    int m;          /* stored correction pairs, 1..10 (10 when <= 0) */
    int max_iter;   /* iterations, >= 0 */
    int max_ls;     /* loss evaluations per line search (20 when <= 0) */
    double pgtol;   /* stop when the largest entry of the projected gradient is <= pgtol (>= 0) */
    double factr;   /* stop when the loss decreases by <= factr * 2.2e-16 relative (>= 0) */
} sr_lbfgsb_cfg;

enum { SR_LBFGSB_PGTOL = 0, SR_LBFGSB_FACTR = 1, SR_LBFGSB_MAX_ITER = 2, SR_LBFGSB_LINE_SEARCH = 3 };

typedef struct {
    int iterations;   /* accepted steps */
    int evaluations;  /* loss-and-gradient evaluations, the first included */
    int status;       /* SR_LBFGSB_*: why it stopped (LINE_SEARCH: no strong-Wolfe step within max_ls) */
    double f;         /* loss at the returned parameters */
    double pg_norm;   /* largest entry of the projected gradient there */
} sr_lbfgsb_info;

/* Minimise the problem's loss from params_dev (device, sr_param_count floats; overwritten with the
 * last accepted iterate, the bounded entries first clipped into their bounds).  f_history: NULL,
 * or a host array of max_iter + 1 doubles receiving the loss of the start and of every iterate.
 * info may be NULL.  Every n-long vector operation runs on the device; the 2m x 2m algebra and
 * the breakpoints of the bounded range (a few thousand values at most) run on the host in FP64.
 * Allocates and frees 2 (m + 1) + 4 vectors of sr_param_count floats; synchronises the stream.
 * Errors as sr_loss_and_grad, SR_ERR_ARG for a bad configuration. */
sr_status sr_lbfgsb(sr_problem *p, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                    sr_lbfgsb_info *info);

/* The same over a batch: L-BFGS-B on the batch's total loss (the sum of its fields' losses) over
 * the packed parameters of sr_batch_param_offset, each field with its own bounds; one batched
 * evaluation per line-search trial.  Arguments and errors as sr_lbfgsb, on the batch's stream. */
sr_status sr_batch_lbfgsb(sr_batch *b, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                          sr_lbfgsb_info *info);

/* Independent L-BFGS-B runs, one per field of the batch (the algorithm and configuration of
 * sr_lbfgsb), advanced together: every iteration builds the direction of each field still running
 * from its own memory of pairs, then runs line-search rounds, each one batched evaluation of all
 * fields, until every running field has its strong-Wolfe step or has used max_ls evaluations; a
 * field stops on its own criteria (its projected gradient, its relative decrease, its iteration
 * count) and keeps its parameters while the others go on.  A field's iterates do not depend on
 * the other fields of the batch.  params_dev: the packed parameters of sr_batch_param_offset
 * (device, overwritten with each field's last accepted iterate, bounded entries clipped first).
 * f_history: NULL or a host array [fields][max_iter + 1] (each field's start and iterates, NaN
 * after its last); info: NULL or a host array of one sr_lbfgsb_info per field; rounds: NULL or
 * receives the number of batched evaluations after the first.  The 2m x 2m algebra and the
 * breakpoints run on the host in FP64, fields in parallel on up to 16 host threads; every n-long
 * operation runs on the device, per field.  Allocates and frees 2 (m + 1) + 5 vectors of the batch's
 * parameter count; synchronises the stream.  Errors as sr_batch_lbfgsb. */
sr_status sr_batch_lbfgsb_fields(sr_batch *b, float *params_dev, const sr_lbfgsb_cfg *cfg, double *f_history,
                                 sr_lbfgsb_info *info, int *rounds);

/* Phase timings of one sr_noise_weights call: CUDA-event durations on its stream, summed over
 * the batches of realisations. */
typedef struct {
    double draw_ms;     /* normal draws divided by sigma_eff */
    double corr_ms;     /* the S_1^T correlation, the dominant kernel */
    double starlet_ms;  /* starlet analysis with the per-coefficient sums */
    double final_ms;    /* the final reductions */
    int launches;       /* kernels the call launched */
    int batch;          /* realisations per batch */
} sr_noise_timing;

/* Prior weights W by Monte Carlo noise propagation (sec. 2.3 and App. B): realisation r draws a
 * standard normal field z_r on the F x F fine grid (F = f N), forms (C^)^-1 dd = z_r / sigma_eff
 * with sigma_eff^-2 = sum_i sigma_i^-2 the co-added noise of the E epochs replicated over each
 * f x f block (sigma = +inf masks a pixel of an epoch), applies S_1^T (the transpose of the
 * zero-padded convolution with epoch 1's narrow PSF, i.e. a correlation) and the starlet
 * analysis with J planes.
 *   sigma_dev  float32 [E][N][N], device; each value > 0 or +inf;
 *   s1_dev     float32 [K][K], device, origin (K/2, K/2), the narrow PSF of epoch 1 (or, for a
 *              PSF fit, the kernel the pixel grid is convolved with);
 *   n_real     realisations (>= 2; the paper uses 5000); seed selects the random stream:
 *              normal number n is Philox4x64-10 block n/4 (counter (n/4, 0, 0, 0), key
 *              (seed, 0)), words (0,1) and (2,3) giving two Box-Muller pairs (cos, sin) from the
 *              24-bit uniforms ((w >> 40) + 1) 2^-24; realisation r takes numbers r F^2 ..
 *              r F^2 + F^2 - 1 in row-major pixel order;
 *   W_host     float32 [J-1], host, or NULL: per detail scale, the sample standard deviation of
 *              all its coefficients of all realisations (the weights sr_set_weights takes);
 *   W_map_dev  float32 [J-1][F][F], device, or NULL: per coefficient, the sample standard
 *              deviation over the realisations; at least one of the two outputs is required;
 *   timing     NULL, or receives the phase timings (the call then synchronises every batch).
 * Arithmetic is FP32; the moments are accumulated in FP64 in a fixed order, so the result does
 * not depend on the run.  The call allocates and frees its workspace (two F x F float buffers
 * per realisation of a batch, at most 64 MB, plus 2 x S x (J-1) x F^2 doubles with S <= 16),
 * orders its work on cuda_stream and synchronises it.  SR_ERR_SHAPE for bad sizes,
 * SR_ERR_UNSUPPORTED for a K whose staging does not fit shared memory (K above about 500),
 * SR_ERR_NONFINITE for a NaN or non-positive sigma or a non-finite s1, SR_ERR_OOM,
 * SR_ERR_CUDA. */
sr_status sr_noise_weights(int N, int f, int K, int J, int E, const float *sigma_dev, const float *s1_dev,
                           int n_real, uint64_t seed, float *W_host, float *W_map_dev, sr_noise_timing *timing,
                           void *cuda_stream);

/* Loss and gradient of one deconvolution field, allocating nothing.
 *
 * The paper has no counterpart to this call: it exists for callers that cannot
 * allocate device memory, neither themselves nor through this library, e.g.
 * code running inside a device-memory pool that was sized once at start-up,
 * a loop that must never block on the allocator, or a host runtime that owns
 * all device memory.  It computes what sr_create_problem + set_* +
 * sr_loss_and_grad compute (folded direct form), but every intermediate buffer
 * (weights, folded PSF kernels, residual and adjoint images, partial sums,
 * starlet planes, work lists) lives in one file-scope device array of
 * SR_NOALLOC_SCRATCH_BYTES (64 MiB), which every GPU that loads the library
 * holds until the process exits.
 *
 * Arguments: desc (DECONV; data_n <= 256; conv_mode AUTO or DIRECT), device
 * pointers d [E][N][N], sigma [E][N][N], psf [E][K][K] and params (packed
 * DECONV layout), host pointer W [J-1]; outputs loss_dev (one device double)
 * and grad_dev (sr_param_count floats, device); cuda_stream orders the work.
 * Sizes whose scratch would exceed SR_NOALLOC_SCRATCH_BYTES are rejected with
 * SR_ERR_SHAPE (the message gives the bytes needed); for config-3-sized fields
 * (300 epochs of 64x64, f = 2, K = 64) about 35 MB are used.
 * The call does not synchronise and returns no input check: NaN data give a
 * NaN loss, and so does any sigma that is NaN or <= 0 (sigma = +inf masks the
 * pixel as elsewhere).  The tile layout (phase groups per output tile) follows
 * the same shared-memory rule as a created problem, so both accept the same
 * shapes.  The first call on a device looks up the
 * array's device address and configures the kernels (under a lock, so first
 * calls from several host threads are safe); make that first call before any
 * stream capture.  Every call uses the same array and leaves the
 * previous call's contents in it; calls whose work overlaps on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller. */
#define SR_NOALLOC_SCRATCH_BYTES (64u << 20)
sr_status sr_loss_and_grad_noalloc(const sr_problem_desc *desc, const float *d_dev, const float *sigma_dev,
                                   const float *psf_dev, const float *W_host, const float *params_dev,
                                   double *loss_dev, float *grad_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* STARRED_H */
