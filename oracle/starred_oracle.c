/*
 * FP64 CPU oracle for the STARRED loss and gradient (Millon et al., arXiv 2402.08725).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product path (the CUDA
 * library and its Python binding) never calls it and shares no code with it.
 *
 * Everything here is written literally, in the paper's operator order, in
 * double precision:
 *   - the model is rasterised at full fine resolution (no truncation of the
 *     Gaussians),
 *   - the narrow-PSF convolution S is the plain double sum over the fine grid,
 *   - D is the plain f x f block sum,
 *   - every adjoint is the explicit transpose of its forward step (scatter
 *     form), not a re-derived gather.
 * It is slow on purpose; a reader can check each function against the cited
 * equation by eye.
 *
 * Conventions (the paper leaves these open; the readings are fixed here):
 *   fine grid F = f*N; arrays are [row][col] row-major; a 2-vector (x, y) has
 *   x along columns.  Fine pixel u has data coordinate (u + 0.5)/f - 0.5; the
 *   stamp centre (N-1)/2 maps to u0 = (F-1)/2, so a source at offset c (data px
 *   from the stamp centre) sits at fine coordinate u0 + f*c.
 *   PSF kernels have odd or even size K with origin o = K/2 (integer division);
 *   S is a true convolution (kernel flipped) with zero padding, output F x F.
 *   D is a flux-conserving block SUM over f x f fine pixels.
 *   The narrow Gaussian r has FWHM 2 fine px (Eq. 1, sec. 2.1), point-sampled:
 *   g(v) = exp(-|v|^2 / (2 sigma^2)) / (2 pi sigma^2), sigma = 1/sqrt(2 ln 2).
 *   The starlet is the isotropic undecimated (a trous) B3-spline transform,
 *   filter [1,4,6,4,1]/16 with holes 2^j at level j, whole-sample mirror borders.
 *   J counts all planes (J-1 detail planes, penalised, plus one coarse plane,
 *   not penalised).
 *   Gamma_i is the spatially constant background of Eq. 9 (sec. 2.2), added
 *   after D as f^2 * Gamma_i per data pixel.
 *   Noise: w = 1/sigma^2 (Eq. 10: C diagonal); sigma = +inf masks a pixel (w = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_in_parallel(void) { return 1; }
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_SHAPE 2
#define ORC_ERR_OOM 5

static const double B3[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};

/* sigma of the narrow Gaussian: FWHM 2 fine px (Eq. 1, sec. 2.1). */
static double gauss_sigma(void) { return 2.0 / (2.0 * sqrt(2.0 * log(2.0))); }

/* 2-D point-sampled unit-flux Gaussian value at offset (vx, vy). */
static double gauss2(double vx, double vy) {
    double s = gauss_sigma();
    return exp(-(vx * vx + vy * vy) / (2.0 * s * s)) / (2.0 * M_PI * s * s);
}

/* 1-D factor of the same Gaussian: gauss2(vx, vy) = gauss1(vx) * gauss1(vy). */
static double gauss1(double v) {
    double s = gauss_sigma();
    return exp(-v * v / (2.0 * s * s)) / (sqrt(2.0 * M_PI) * s);
}

static int orc_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_version(void) { return 1; }

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of later calls (timing only: every reduction runs in a fixed order, so the results do
   not depend on it). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* S: narrow-PSF convolution on the fine grid (Eq. 8 and Eq. 10, sec. 2.2).  */
/* ------------------------------------------------------------------------- */

/* out[u] = sum_q s[q] * x[u - q + o], zero outside [0,F)^2, o = K/2.
 * Output rows are independent; when not already inside a parallel region they are
 * shared among threads (each pixel's sum keeps its order, so results do not change). */
int orc_conv_same(int F, int K, const double *x, const double *s, double *out) {
    if (F <= 0 || K <= 0) return ORC_ERR_SHAPE;
    int o = K / 2;
#pragma omp parallel for schedule(static) if (!omp_in_parallel() && (long)F * F * K * K > 100000000L)
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double acc = 0.0;
            for (int qy = 0; qy < K; ++qy) {
                int y = uy - qy + o;
                if (y < 0 || y >= F) continue;
                for (int qx = 0; qx < K; ++qx) {
                    int xx = ux - qx + o;
                    if (xx < 0 || xx >= F) continue;
                    acc += s[qy * K + qx] * x[y * F + xx];
                }
            }
            out[uy * F + ux] = acc;
        }
    return ORC_OK;
}

/* Scatter of the rows [uy0, uy1) of y into out (added). */
static void conv_adjoint_rows(int F, int K, int uy0, int uy1, const double *y, const double *s, double *out) {
    int o = K / 2;
    for (int uy = uy0; uy < uy1; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double yu = y[uy * F + ux];
            if (yu == 0.0) continue;
            for (int qy = 0; qy < K; ++qy) {
                int vy = uy - qy + o;
                if (vy < 0 || vy >= F) continue;
                for (int qx = 0; qx < K; ++qx) {
                    int vx = ux - qx + o;
                    if (vx < 0 || vx >= F) continue;
                    out[vy * F + vx] += s[qy * K + qx] * yu;
                }
            }
        }
}

/* Transpose of orc_conv_same, written as the scatter of each forward term:
 * every term s[q]*x[u-q+o] of out[u] sends s[q]*y[u] to position u-q+o.
 * Large sizes scatter a fixed number of row bands into private images, summed in band
 * order (the same result for any number of threads). */
int orc_conv_same_adjoint(int F, int K, const double *y, const double *s, double *out) {
    if (F <= 0 || K <= 0) return ORC_ERR_SHAPE;
    memset(out, 0, sizeof(double) * (size_t)F * F);
    const int bands = 16;
    size_t n = (size_t)F * F;
    if (omp_in_parallel() || (long)F * F * K * K <= 100000000L || F < bands) {
        conv_adjoint_rows(F, K, 0, F, y, s, out);
        return ORC_OK;
    }
    double *part = calloc(n * bands, sizeof(double));
    if (!part) return ORC_ERR_OOM;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < bands; ++b)
        conv_adjoint_rows(F, K, (int)((long)F * b / bands), (int)((long)F * (b + 1) / bands), y, s, part + n * b);
    for (int b = 0; b < bands; ++b)
        for (size_t k = 0; k < n; ++k) out[k] += part[n * b + k];
    free(part);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* D: block-sum downsampling (the subsampling arrow of Eq. 1) and its adjoint */
/* ------------------------------------------------------------------------- */

int orc_downsample(int N, int f, const double *x, double *out) {
    if (N <= 0 || f <= 0) return ORC_ERR_SHAPE;
    int F = f * N;
    for (int py = 0; py < N; ++py)
        for (int px = 0; px < N; ++px) {
            double acc = 0.0;
            for (int a = 0; a < f; ++a)
                for (int b = 0; b < f; ++b) acc += x[(f * py + a) * F + (f * px + b)];
            out[py * N + px] = acc;
        }
    return ORC_OK;
}

/* D^T: each data pixel's value is sent to every fine pixel of its block. */
int orc_downsample_adjoint(int N, int f, const double *e, double *out) {
    if (N <= 0 || f <= 0) return ORC_ERR_SHAPE;
    int F = f * N;
    memset(out, 0, sizeof(double) * (size_t)F * F);
    for (int py = 0; py < N; ++py)
        for (int px = 0; px < N; ++px)
            for (int a = 0; a < f; ++a)
                for (int b = 0; b < f; ++b) out[(f * py + a) * F + (f * px + b)] += e[py * N + px];
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Starlet transform Phi^T (Eq. 6, sec. 2.1): B3-spline a trous, mirror borders */
/* ------------------------------------------------------------------------- */

static int mirror(int t, int F) {
    if (t < 0) return -t;
    if (t > F - 1) return 2 * (F - 1) - t;
    return t;
}

int orc_starlet_valid(int F, int J) {
    if (J < 2 || F < 2) return 0;
    /* widest hole used is 2 * 2^(J-2); single-bounce mirroring needs it <= F-1 */
    return 2 * (1 << (J - 2)) <= F - 1;
}

/* out = H_j x: separable smoothing with holes 2^j, rows first then columns. */
static void starlet_smooth(int F, int j, const double *x, double *tmp, double *out) {
    int step = 1 << j;
    for (int y = 0; y < F; ++y)
        for (int xx = 0; xx < F; ++xx) {
            double acc = 0.0;
            for (int n = -2; n <= 2; ++n) acc += B3[n + 2] * x[y * F + mirror(xx + n * step, F)];
            tmp[y * F + xx] = acc;
        }
    for (int y = 0; y < F; ++y)
        for (int xx = 0; xx < F; ++xx) {
            double acc = 0.0;
            for (int m = -2; m <= 2; ++m) acc += B3[m + 2] * tmp[mirror(y + m * step, F) * F + xx];
            out[y * F + xx] = acc;
        }
}

/* out = H_j^T y, as the scatter transpose of the column pass then of the row pass. */
static void starlet_smooth_adjoint(int F, int j, const double *y, double *tmp, double *out) {
    int step = 1 << j;
    memset(tmp, 0, sizeof(double) * (size_t)F * F);
    for (int r = 0; r < F; ++r)
        for (int xx = 0; xx < F; ++xx)
            for (int m = -2; m <= 2; ++m) tmp[mirror(r + m * step, F) * F + xx] += B3[m + 2] * y[r * F + xx];
    memset(out, 0, sizeof(double) * (size_t)F * F);
    for (int r = 0; r < F; ++r)
        for (int xx = 0; xx < F; ++xx)
            for (int n = -2; n <= 2; ++n) out[r * F + mirror(xx + n * step, F)] += B3[n + 2] * tmp[r * F + xx];
}

/* Analysis A: out[0..J-2] = detail planes w_1..w_{J-1}, out[J-1] = coarse c_{J-1}.
 * c_0 = h, c_{j+1} = H_j c_j, w_{j+1} = c_j - c_{j+1}. */
int orc_starlet_analysis(int F, int J, const double *h, double *out) {
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t n = (size_t)F * F;
    double *c = malloc(sizeof(double) * n), *cn = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    if (!c || !cn || !tmp) { free(c); free(cn); free(tmp); return ORC_ERR_OOM; }
    memcpy(c, h, sizeof(double) * n);
    for (int j = 0; j < J - 1; ++j) {
        starlet_smooth(F, j, c, tmp, cn);
        for (size_t k = 0; k < n; ++k) out[(size_t)j * n + k] = c[k] - cn[k];
        memcpy(c, cn, sizeof(double) * n);
    }
    memcpy(out + (size_t)(J - 1) * n, c, sizeof(double) * n);
    free(c); free(cn); free(tmp);
    return ORC_OK;
}

/* Adjoint A^T of orc_starlet_analysis: y[0..J-2] pair with w_1..w_{J-1},
 * y[J-1] with the coarse plane.  With T_j the gradient reaching c_j through
 * w_{j+1} and c_{j+1}:  T_{J-1} = y_coarse,
 * T_j = y_{j+1} + H_j^T (T_{j+1} - y_{j+1}),  A^T y = T_0. */
int orc_starlet_adjoint(int F, int J, const double *y, double *out) {
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t n = (size_t)F * F;
    double *T = malloc(sizeof(double) * n), *v = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
    if (!T || !v || !tmp) { free(T); free(v); free(tmp); return ORC_ERR_OOM; }
    memcpy(T, y + (size_t)(J - 1) * n, sizeof(double) * n);
    for (int j = J - 2; j >= 0; --j) {
        const double *yj = y + (size_t)j * n; /* pairs with w_{j+1} */
        for (size_t k = 0; k < n; ++k) v[k] = T[k] - yj[k];
        starlet_smooth_adjoint(F, j, v, tmp, T);
        for (size_t k = 0; k < n; ++k) T[k] += yj[k];
    }
    memcpy(out, T, sizeof(double) * n);
    free(T); free(v); free(tmp);
    return ORC_OK;
}

/* Prior P = lambda * sum_{j=1}^{J-1} W_j * sum_u |w_j[u]| (Eq. 6 / Eq. 11),
 * one weight per detail scale.  Returns P; writes dP/dh into grad (if not NULL),
 * with the subgradient sign(0) = 0. */
int orc_starlet_prior(int F, int J, double lam, const double *W, const double *h, double *prior, double *grad) {
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t n = (size_t)F * F;
    double *planes = malloc(sizeof(double) * n * J);
    if (!planes) return ORC_ERR_OOM;
    int rc = orc_starlet_analysis(F, J, h, planes);
    if (rc) { free(planes); return rc; }
    double p = 0.0;
    for (int j = 0; j < J - 1; ++j) {
        double sj = 0.0;
        for (size_t k = 0; k < n; ++k) sj += fabs(planes[(size_t)j * n + k]);
        p += lam * W[j] * sj;
    }
    *prior = p;
    if (grad) {
        /* y_j = lambda W_j sign(w_j) for detail planes, 0 for the coarse plane */
        for (int j = 0; j < J - 1; ++j)
            for (size_t k = 0; k < n; ++k) {
                double w = planes[(size_t)j * n + k];
                planes[(size_t)j * n + k] = lam * W[j] * (w > 0 ? 1.0 : (w < 0 ? -1.0 : 0.0));
            }
        memset(planes + (size_t)(J - 1) * n, 0, sizeof(double) * n);
        rc = orc_starlet_adjoint(F, J, planes, grad);
    }
    free(planes);
    return rc;
}

/* The prior with one weight per coefficient (sec. 2.3 and App. B propagate the noise to a map per
 * scale; the paper then takes one value per scale, R15): lambda sum_j sum_u Wmap[j][u] |w_j(u)|
 * over the J - 1 detail planes, Wmap [J-1][F][F]; gradient A^T (lambda Wmap o sign(A h)). */
int orc_starlet_prior_map(int F, int J, double lam, const double *Wmap, const double *h, double *prior,
                          double *grad) {
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t n = (size_t)F * F;
    double *planes = malloc(sizeof(double) * n * J);
    if (!planes) return ORC_ERR_OOM;
    int rc = orc_starlet_analysis(F, J, h, planes);
    if (rc) { free(planes); return rc; }
    double p = 0.0;
    for (int j = 0; j < J - 1; ++j)
        for (size_t k = 0; k < n; ++k) p += lam * Wmap[(size_t)j * n + k] * fabs(planes[(size_t)j * n + k]);
    *prior = p;
    if (grad) {
        for (int j = 0; j < J - 1; ++j)
            for (size_t k = 0; k < n; ++k) {
                double w = planes[(size_t)j * n + k];
                planes[(size_t)j * n + k] = lam * Wmap[(size_t)j * n + k] * (w > 0 ? 1.0 : (w < 0 ? -1.0 : 0.0));
            }
        memset(planes + (size_t)(J - 1) * n, 0, sizeof(double) * n);
        rc = orc_starlet_adjoint(F, J, planes, grad);
    }
    free(planes);
    return rc;
}

/* The prior with per-scale weights W, or with the per-coefficient map Wmap when it is not NULL. */
static int prior_w(int F, int J, double lam, const double *W, const double *Wmap, const double *h, double *prior,
                   double *grad) {
    return Wmap ? orc_starlet_prior_map(F, J, lam, Wmap, h, prior, grad) : orc_starlet_prior(F, J, lam, W, h, prior, grad);
}

/* ------------------------------------------------------------------------- */
/* Point-source channel (Eq. 9, sec. 2.2; r_k of Eq. 3)                       */
/* ------------------------------------------------------------------------- */

/* out[u] += amp * g(u - (ux_c, uy_c)) over the whole fine grid. */
int orc_add_gaussian(int F, double amp, double ux_c, double uy_c, double *out) {
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) out[uy * F + ux] += amp * gauss2(ux - ux_c, uy - uy_c);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Joint multi-epoch deconvolution: loss Eq. 11 (lambda_pts = 0), Eq. 9, 10   */
/* ------------------------------------------------------------------------- */

/* Packed parameters: [h F*F | a E*M | c M*2 | delta E*2 | Gamma E]. */
static void deconv_offsets(int E, int N, int f, int M, size_t *oh, size_t *oa, size_t *oc, size_t *od, size_t *og,
                           size_t *total) {
    size_t F = (size_t)f * N;
    *oh = 0;
    *oa = F * F;
    *oc = *oa + (size_t)E * M;
    *od = *oc + (size_t)M * 2;
    *og = *od + (size_t)E * 2;
    *total = *og + (size_t)E;
}

size_t orc_deconv_param_count(int E, int N, int f, int M) {
    size_t oh, oa, oc, od, og, t;
    deconv_offsets(E, N, f, M, &oh, &oa, &oc, &od, &og, &t);
    return t;
}

/* Fine coordinate of point source k in epoch i: u0 + f * (c_k + delta_i). */
static void source_centre(int F, int f, const double *c, const double *dl, int k, int i, double *ux, double *uy) {
    double u0 = 0.5 * (F - 1);
    *ux = u0 + f * (c[2 * k + 0] + dl[2 * i + 0]);
    *uy = u0 + f * (c[2 * k + 1] + dl[2 * i + 1]);
}

/* Translation of the fine image h by (sx, sy) fine pixels (the extended channel moved with the
 * epoch's shift, f * delta_i): out(u) = h(u - s) with bilinear interpolation between the four
 * fine pixels around u - s and zero outside the grid.  The paper leaves the interpolation open
 * (sec. 5 names shifts between frames); bilinear is the reading taken. */
static double bilinear_at(int F, const double *h, double px, double py) {
    double fx = floor(px), fy = floor(py);
    int x0 = (int)fx, y0 = (int)fy;
    double tx = px - fx, ty = py - fy, acc = 0.0;
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            int x = x0 + a, y = y0 + b;
            if (x < 0 || x >= F || y < 0 || y >= F) continue;
            acc += (a ? tx : 1.0 - tx) * (b ? ty : 1.0 - ty) * h[(size_t)y * F + x];
        }
    return acc;
}

int orc_translate(int F, double sx, double sy, const double *h, double *out) {
    if (F <= 0) return ORC_ERR_SHAPE;
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) out[(size_t)uy * F + ux] = bilinear_at(F, h, ux - sx, uy - sy);
    return ORC_OK;
}

/* Transpose of orc_translate: every output pixel u scatters its value to the four pixels its
 * interpolation read, with the same weights. */
int orc_translate_adjoint(int F, double sx, double sy, const double *g, double *out) {
    if (F <= 0) return ORC_ERR_SHAPE;
    memset(out, 0, sizeof(double) * (size_t)F * F);
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double px = ux - sx, py = uy - sy, fx = floor(px), fy = floor(py);
            int x0 = (int)fx, y0 = (int)fy;
            double tx = px - fx, ty = py - fy, gv = g[(size_t)uy * F + ux];
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int x = x0 + a, y = y0 + b;
                    if (x < 0 || x >= F || y < 0 || y >= F) continue;
                    out[(size_t)y * F + x] += (a ? tx : 1.0 - tx) * (b ? ty : 1.0 - ty) * gv;
                }
        }
    return ORC_OK;
}

/* d out(u) / d sx and d out(u) / d sy of orc_translate (the derivative of the interpolant inside
 * its cell: minus the weighted differences of the four pixels along each axis). */
static void translate_dshift(int F, double sx, double sy, const double *h, double *dx, double *dy) {
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double px = ux - sx, py = uy - sy, fx = floor(px), fy = floor(py);
            int x0 = (int)fx, y0 = (int)fy;
            double tx = px - fx, ty = py - fy;
            double v[2][2];
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int x = x0 + a, y = y0 + b;
                    v[b][a] = (x < 0 || x >= F || y < 0 || y >= F) ? 0.0 : h[(size_t)y * F + x];
                }
            dx[(size_t)uy * F + ux] = -((1.0 - ty) * (v[0][1] - v[0][0]) + ty * (v[1][1] - v[1][0]));
            dy[(size_t)uy * F + ux] = -((1.0 - tx) * (v[1][0] - v[0][0]) + tx * (v[1][1] - v[0][1]));
        }
}

/* Rotation of an epoch's frame (sec. 5 names rotations between frames; no equation in the paper,
 * so the reading here): the reference-frame point q lands at u = u0 + R (q - u0) + s in the epoch's
 * fine grid, R = [[cos t, -sin t], [sin t, cos t]] acting on (x, y), u0 = (F - 1)/2 the grid centre
 * and s the shift (f delta_i when the extended channel moves with the shifts, else 0).  The epoch
 * sees out(u) = h at q(u) = u0 + R^T (u - u0 - s), bilinear between the four fine pixels around q
 * and zero outside the grid; its point sources sit at u0 + f (R c_k + delta_i). */
static void warp_point(int F, double ct, double st, double sx, double sy, int ux, int uy, double *qx, double *qy) {
    const double u0 = 0.5 * (F - 1), dx = ux - u0 - sx, dy = uy - u0 - sy;
    *qx = u0 + ct * dx + st * dy;
    *qy = u0 - st * dx + ct * dy;
}

int orc_warp(int F, double theta, double sx, double sy, const double *h, double *out) {
    if (F <= 0) return ORC_ERR_SHAPE;
    const double ct = cos(theta), st = sin(theta);
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double qx, qy;
            warp_point(F, ct, st, sx, sy, ux, uy, &qx, &qy);
            out[(size_t)uy * F + ux] = bilinear_at(F, h, qx, qy);
        }
    return ORC_OK;
}

/* Transpose of orc_warp: every output pixel scatters its value to the four pixels it read. */
int orc_warp_adjoint(int F, double theta, double sx, double sy, const double *g, double *out) {
    if (F <= 0) return ORC_ERR_SHAPE;
    const double ct = cos(theta), st = sin(theta);
    memset(out, 0, sizeof(double) * (size_t)F * F);
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double qx, qy;
            warp_point(F, ct, st, sx, sy, ux, uy, &qx, &qy);
            const double fx = floor(qx), fy = floor(qy), tx = qx - fx, ty = qy - fy, gv = g[(size_t)uy * F + ux];
            const int x0 = (int)fx, y0 = (int)fy;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int x = x0 + a, y = y0 + b;
                    if (x < 0 || x >= F || y < 0 || y >= F) continue;
                    out[(size_t)y * F + x] += (a ? tx : 1.0 - tx) * (b ? ty : 1.0 - ty) * gv;
                }
        }
    return ORC_OK;
}

/* d out(u) / d s of orc_warp: q moves by -R^T ds, so d out / d s = -R grad H(q), grad H the
 * derivative of the interpolant inside its cell. */
static void warp_dshift(int F, double theta, double sx, double sy, const double *h, double *dx, double *dy) {
    const double ct = cos(theta), st = sin(theta);
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double qx, qy;
            warp_point(F, ct, st, sx, sy, ux, uy, &qx, &qy);
            const double fx = floor(qx), fy = floor(qy), tx = qx - fx, ty = qy - fy;
            const int x0 = (int)fx, y0 = (int)fy;
            double v[2][2];
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int x = x0 + a, y = y0 + b;
                    v[b][a] = (x < 0 || x >= F || y < 0 || y >= F) ? 0.0 : h[(size_t)y * F + x];
                }
            const double hx = (1.0 - ty) * (v[0][1] - v[0][0]) + ty * (v[1][1] - v[1][0]);
            const double hy = (1.0 - tx) * (v[1][0] - v[0][0]) + tx * (v[1][1] - v[0][1]);
            dx[(size_t)uy * F + ux] = -(ct * hx - st * hy);
            dy[(size_t)uy * F + ux] = -(st * hx + ct * hy);
        }
}

/* Fine centre of point source k in epoch i of a rotated frame: u0 + f (R c_k + delta_i). */
static void source_centre_rot(int F, int f, const double *c, const double *dl, int k, int i, double theta, double *ux,
                              double *uy) {
    const double u0 = 0.5 * (F - 1), ct = cos(theta), st = sin(theta);
    const double cx = c[2 * k + 0], cy = c[2 * k + 1];
    *ux = u0 + f * ((ct * cx - st * cy) + dl[2 * i + 0]);
    *uy = u0 + f * ((st * cx + ct * cy) + dl[2 * i + 1]);
}

/* Model of epoch i on the data grid: M_i = D S_i (h + sum_k a_ki r_k) + f^2 Gamma_i. */
static void deconv_model_epoch(int i, int N, int f, int K, int M, const double *s_i, const double *params,
                               size_t oa, size_t oc, size_t od, size_t og, double *fimg, double *conv, double *model,
                               int translate, const double *theta) {
    int F = f * N;
    size_t n = (size_t)F * F;
    if (theta) /* h seen in the epoch's rotated (and, when translating, shifted) frame */
        orc_warp(F, theta[i], translate ? f * params[od + 2 * (size_t)i] : 0.0,
                 translate ? f * params[od + 2 * (size_t)i + 1] : 0.0, params, fimg);
    else if (translate) /* h moved by the epoch's shift f * delta_i */
        orc_translate(F, f * params[od + 2 * (size_t)i], f * params[od + 2 * (size_t)i + 1], params, fimg);
    else
        memcpy(fimg, params, sizeof(double) * n); /* h */
    for (int k = 0; k < M; ++k) {
        double ux, uy;
        if (theta)
            source_centre_rot(F, f, params + oc, params + od, k, i, theta[i], &ux, &uy);
        else
            source_centre(F, f, params + oc, params + od, k, i, &ux, &uy);
        orc_add_gaussian(F, params[oa + (size_t)i * M + k], ux, uy, fimg);
    }
    orc_conv_same(F, K, fimg, s_i, conv);
    orc_downsample(N, f, conv, model);
    double bg = (double)f * f * params[og + i];
    for (int p = 0; p < N * N; ++p) model[p] += bg;
}

static int deconv_model(int E, int N, int f, int K, int M, const double *s, const double *params, double *model_out,
                        int translate, const double *theta) {
    if (E <= 0 || N <= 0 || f <= 0 || K <= 0 || M < 0) return ORC_ERR_SHAPE;
    int F = f * N;
    size_t oh, oa, oc, od, og, tot;
    deconv_offsets(E, N, f, M, &oh, &oa, &oc, &od, &og, &tot);
    size_t n = (size_t)F * F;
    int err = 0;
    int nt = orc_threads(0);
    if (nt > E) nt = E;
#pragma omp parallel num_threads(nt)
    {
        double *fimg = malloc(sizeof(double) * n), *conv = malloc(sizeof(double) * n);
        if (!fimg || !conv) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(static)
            for (int i = 0; i < E; ++i)
                deconv_model_epoch(i, N, f, K, M, s + (size_t)i * K * K, params, oa, oc, od, og, fimg, conv,
                                   model_out + (size_t)i * N * N, translate, theta);
        }
        free(fimg); free(conv);
    }
    return err ? ORC_ERR_OOM : ORC_OK;
}

static double inv_var(double sigma) { return isinf(sigma) ? 0.0 : 1.0 / (sigma * sigma); }

int orc_deconv_model(int E, int N, int f, int K, int M, const double *s, const double *params, double *model_out) {
    return deconv_model(E, N, f, K, M, s, params, model_out, 0, NULL);
}

/* The model with the frame variants: translate moves h by f delta_i, theta (NULL: none) rotates
 * epoch i's frame by theta[i] radians (warp_point). */
int orc_deconv_model_ex(int E, int N, int f, int K, int M, const double *s, const double *params, double *model_out,
                        int translate, const double *theta) {
    return deconv_model(E, N, f, K, M, s, params, model_out, translate, theta);
}

/* Loss and gradient of the deconvolution problem.
 *   parts[0] = chi^2 term (Eq. 10), parts[1] = starlet prior on h (Eq. 11, first
 *   prior term), loss = parts[0] + parts[1].
 *   grad (nullable) is d loss / d params in the packed layout.
 *   chi2_epoch (nullable) receives the chi^2 of each epoch. */
static int deconv_loss_grad(int E, int N, int f, int K, int M, int J, double lam, const double *d,
                            const double *sigma, const double *s, const double *W, const double *params, double *parts,
                            double *grad, double *chi2_epoch, int nthreads, int translate, const double *theta,
                            const double *Wmap) {
    if (E <= 0 || N <= 0 || f <= 0 || K <= 0 || M < 0) return ORC_ERR_SHAPE;
    int F = f * N;
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t oh, oa, oc, od, og, tot;
    deconv_offsets(E, N, f, M, &oh, &oa, &oc, &od, &og, &tot);
    size_t n = (size_t)F * F;
    int nt = orc_threads(nthreads);
    if (nt > E) nt = E; /* fewer epochs than threads: the convolutions share the rest */
    double *chi = calloc((size_t)E, sizeof(double));
    /* per-epoch gradient wrt the fine image f_i, summed into dh afterwards in epoch order */
    double *gfine = grad ? malloc(sizeof(double) * n * (size_t)E) : NULL;
    /* d loss / d (fine centre of source k in epoch i), reduced in fixed order below */
    double *dcen = grad ? calloc((size_t)E * M * 2 + 1, sizeof(double)) : NULL;
    double *dshift = grad ? calloc((size_t)E * 2, sizeof(double)) : NULL;
    if (!chi || (grad && (!gfine || !dcen || !dshift))) {
        free(chi); free(gfine); free(dcen); free(dshift);
        return ORC_ERR_OOM;
    }
    if (grad) memset(grad, 0, sizeof(double) * tot);
    const double sg = gauss_sigma();
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        double *fimg = malloc(sizeof(double) * n), *conv = malloc(sizeof(double) * n);
        double *model = malloc(sizeof(double) * (size_t)N * N), *e = malloc(sizeof(double) * (size_t)N * N);
        double *ey = malloc(sizeof(double) * n);
        if (!fimg || !conv || !model || !e || !ey) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int i = 0; i < E; ++i) {
                const double *s_i = s + (size_t)i * K * K;
                deconv_model_epoch(i, N, f, K, M, s_i, params, oa, oc, od, og, fimg, conv, model, translate, theta);
                double c2 = 0.0;
                for (int p = 0; p < N * N; ++p) {
                    size_t ip = (size_t)i * N * N + p;
                    double w = inv_var(sigma[ip]);
                    double r = d[ip] - model[p];
                    c2 += 0.5 * w * r * r;
                    e[p] = -w * r; /* d chi^2 / d model */
                }
                chi[i] = c2;
                if (!grad) continue;
                /* dGamma_i = f^2 sum_p e_p */
                double se = 0.0;
                for (int p = 0; p < N * N; ++p) se += e[p];
                grad[og + i] = (double)f * f * se;
                /* d chi^2 / d f_i = S_i^T D^T e */
                orc_downsample_adjoint(N, f, e, ey);
                double *G = gfine + (size_t)i * n;
                orc_conv_same_adjoint(F, K, ey, s_i, G);
                /* point sources: d/da_ki and d/d(centre) through the Gaussian */
                for (int k = 0; k < M; ++k) {
                    double ux, uy;
                    if (theta)
                        source_centre_rot(F, f, params + oc, params + od, k, i, theta[i], &ux, &uy);
                    else
                        source_centre(F, f, params + oc, params + od, k, i, &ux, &uy);
                    double aki = params[oa + (size_t)i * M + k];
                    double ga = 0.0, gx = 0.0, gy = 0.0;
                    for (int vy = 0; vy < F; ++vy)
                        for (int vx = 0; vx < F; ++vx) {
                            double gv = gauss2(vx - ux, vy - uy);
                            double Gv = G[vy * F + vx];
                            ga += Gv * gv;
                            /* d g(v - u_c) / d u_c = g * (v - u_c) / sigma^2 */
                            gx += Gv * gv * (vx - ux) / (sg * sg);
                            gy += Gv * gv * (vy - uy) / (sg * sg);
                        }
                    grad[oa + (size_t)i * M + k] = ga;
                    dcen[((size_t)i * M + k) * 2 + 0] = aki * gx;
                    dcen[((size_t)i * M + k) * 2 + 1] = aki * gy;
                }
                if (translate) {
                    /* the moved h: d/d delta_i = f sum_u G(u) d(T h)(u)/d s (conv and ey as scratch) */
                    const double sx = f * params[od + 2 * (size_t)i], sy = f * params[od + 2 * (size_t)i + 1];
                    if (theta)
                        warp_dshift(F, theta[i], sx, sy, params, conv, ey);
                    else
                        translate_dshift(F, sx, sy, params, conv, ey);
                    double tx = 0.0, ty = 0.0;
                    for (size_t u = 0; u < n; ++u) {
                        tx += G[u] * conv[u];
                        ty += G[u] * ey[u];
                    }
                    dshift[2 * (size_t)i + 0] = f * tx;
                    dshift[2 * (size_t)i + 1] = f * ty;
                }
            }
        }
        free(fimg); free(conv); free(model); free(e); free(ey);
    }
    if (err) { free(chi); free(gfine); free(dcen); free(dshift); return ORC_ERR_OOM; }
    if (grad) {
        /* fine centre = u0 + f (R_i c_k + delta_i): the chain factor of delta_i is f, of c_k f R_i^T */
        for (int i = 0; i < E; ++i)
            for (int k = 0; k < M; ++k) {
                const double vx = f * dcen[((size_t)i * M + k) * 2 + 0], vy = f * dcen[((size_t)i * M + k) * 2 + 1];
                if (theta) {
                    const double ct = cos(theta[i]), st = sin(theta[i]);
                    grad[oc + 2 * k + 0] += ct * vx + st * vy;
                    grad[oc + 2 * k + 1] += -st * vx + ct * vy;
                } else {
                    grad[oc + 2 * k + 0] += vx;
                    grad[oc + 2 * k + 1] += vy;
                }
                grad[od + 2 * i + 0] += vx;
                grad[od + 2 * i + 1] += vy;
            }
        if (translate)
            for (int i = 0; i < E; ++i)
                for (int ax = 0; ax < 2; ++ax) grad[od + 2 * i + ax] += dshift[2 * i + ax];
    }
    free(dcen); free(dshift);
    double chi2 = 0.0;
    for (int i = 0; i < E; ++i) chi2 += chi[i];
    if (chi2_epoch) memcpy(chi2_epoch, chi, sizeof(double) * E);
    double prior = 0.0;
    double *gprior = grad ? malloc(sizeof(double) * n) : NULL;
    int rc = prior_w(F, J, lam, W, Wmap, params + oh, &prior, gprior);
    if (grad && rc == ORC_OK && (translate || theta)) {
        /* d/dh = sum_i T_i^T G_i (epochs in order), plus the prior's part */
        double *tg = malloc(sizeof(double) * n);
        if (!tg) rc = ORC_ERR_OOM;
        for (size_t u = 0; tg && u < n; ++u) grad[oh + u] = gprior[u];
        for (int i = 0; tg && i < E; ++i) {
            const double sx = translate ? f * params[od + 2 * (size_t)i] : 0.0;
            const double sy = translate ? f * params[od + 2 * (size_t)i + 1] : 0.0;
            if (theta)
                orc_warp_adjoint(F, theta[i], sx, sy, gfine + (size_t)i * n, tg);
            else
                orc_translate_adjoint(F, sx, sy, gfine + (size_t)i * n, tg);
            for (size_t u = 0; u < n; ++u) grad[oh + u] += tg[u];
        }
        free(tg);
    } else if (grad && rc == ORC_OK) {
        for (size_t u = 0; u < n; ++u) {
            double acc = gprior[u];
            for (int i = 0; i < E; ++i) acc += gfine[(size_t)i * n + u];
            grad[oh + u] = acc;
        }
    }
    parts[0] = chi2;
    parts[1] = prior;
    free(gprior); free(chi); free(gfine);
    return rc;
}

int orc_deconv_loss_grad(int E, int N, int f, int K, int M, int J, double lam, const double *d, const double *sigma,
                         const double *s, const double *W, const double *params, double *parts, double *grad,
                         double *chi2_epoch, int nthreads) {
    return deconv_loss_grad(E, N, f, K, M, J, lam, d, sigma, s, W, params, parts, grad, chi2_epoch, nthreads, 0, NULL,
                            NULL);
}

/* The same with the extended channel moved by each epoch's shift: f_i = T_{f delta_i} h + P_i
 * (orc_translate); the gradient of delta_i then also has the moved h's part. */
int orc_deconv_loss_grad_shifted(int E, int N, int f, int K, int M, int J, double lam, const double *d,
                                 const double *sigma, const double *s, const double *W, const double *params,
                                 double *parts, double *grad, double *chi2_epoch, int nthreads) {
    return deconv_loss_grad(E, N, f, K, M, J, lam, d, sigma, s, W, params, parts, grad, chi2_epoch, nthreads, 1, NULL,
                            NULL);
}

/* The same with the frame variants of orc_deconv_model_ex: translate (0 or 1) and theta (NULL or
 * [E] rotation angles in radians, fixed inputs: no gradient); Wmap (NULL or [J-1][F][F]) weights
 * each starlet coefficient of the prior on its own (orc_starlet_prior_map) instead of W. */
int orc_deconv_loss_grad_ex(int E, int N, int f, int K, int M, int J, double lam, const double *d, const double *sigma,
                            const double *s, const double *W, const double *params, double *parts, double *grad,
                            double *chi2_epoch, int nthreads, int translate, const double *theta, const double *Wmap) {
    return deconv_loss_grad(E, N, f, K, M, J, lam, d, sigma, s, W, params, parts, grad, chi2_epoch, nthreads,
                            translate, theta, Wmap);
}

/* Point-source prior, the third term of Eq. 11 (sec. 2.2):
 *   lambda_pts || W o Phi^T sum_k <a_k> r_k ||_1,   <a_k> = (1/E) sum_i a_ki,
 * with r_k the unit Gaussian of Eq. 1 at the source's centre c_k (no per-epoch shift: the
 * term regularises the mean point-source image).  *value receives the term; when grad is not
 * NULL its gradient is ADDED to the a and c blocks of grad (packed deconvolution layout):
 *   d/da_ki = (1/E) sum_u G[u] r_k[u],
 *   d/dc_k  = <a_k> sum_u G[u] d r_k[u] / d c_k,  d r_k / d c_k = f (u - centre_k) / s^2 r_k,
 * G = Phi (lambda_pts W o sign(Phi^T P)) the prior's gradient with respect to the image P. */
static int pts_prior(int E, int N, int f, int M, int J, double lam_pts, const double *W, const double *Wmap,
                     const double *params, double *value, double *grad) {
    if (E <= 0 || N <= 0 || f <= 0 || M < 0) return ORC_ERR_SHAPE;
    const int F = f * N;
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t oh, oa, oc, od, og, tot;
    deconv_offsets(E, N, f, M, &oh, &oa, &oc, &od, &og, &tot);
    const size_t n = (size_t)F * F;
    double *P = calloc(n, sizeof(double)), *G = malloc(sizeof(double) * n), *abar = calloc((size_t)M + 1, sizeof(double));
    double *zero = calloc(2, sizeof(double));
    if (!P || !G || !abar || !zero) { free(P); free(G); free(abar); free(zero); return ORC_ERR_OOM; }
    for (int k = 0; k < M; ++k) {
        for (int i = 0; i < E; ++i) abar[k] += params[oa + (size_t)i * M + k];
        abar[k] /= E;
        double ux, uy;
        source_centre(F, f, params + oc, zero, k, 0, &ux, &uy);
        orc_add_gaussian(F, abar[k], ux, uy, P);
    }
    int rc = prior_w(F, J, lam_pts, W, Wmap, P, value, grad ? G : NULL);
    if (rc == ORC_OK && grad) {
        const double s2 = gauss_sigma() * gauss_sigma();
        for (int k = 0; k < M; ++k) {
            double ux, uy;
            source_centre(F, f, params + oc, zero, k, 0, &ux, &uy);
            double sa = 0.0, sx = 0.0, sy = 0.0;
            for (int vy = 0; vy < F; ++vy)
                for (int vx = 0; vx < F; ++vx) {
                    const double g = gauss2(vx - ux, vy - uy), Gv = G[(size_t)vy * F + vx];
                    sa += Gv * g;
                    sx += Gv * g * (vx - ux) / s2;
                    sy += Gv * g * (vy - uy) / s2;
                }
            for (int i = 0; i < E; ++i) grad[oa + (size_t)i * M + k] += sa / E;
            grad[oc + 2 * k + 0] += abar[k] * f * sx;
            grad[oc + 2 * k + 1] += abar[k] * f * sy;
        }
    }
    free(P); free(G); free(abar); free(zero);
    return rc;
}

int orc_pts_prior(int E, int N, int f, int M, int J, double lam_pts, const double *W, const double *params,
                  double *value, double *grad) {
    return pts_prior(E, N, f, M, J, lam_pts, W, NULL, params, value, grad);
}

/* The point-source prior with the per-coefficient weights Wmap [J-1][F][F]. */
int orc_pts_prior_map(int E, int N, int f, int M, int J, double lam_pts, const double *Wmap, const double *params,
                      double *value, double *grad) {
    return pts_prior(E, N, f, M, J, lam_pts, NULL, Wmap, params, value, grad);
}

/* Weighted L1 norm of the detail planes, sum_j W_j || (Phi^T x)_j ||_1. */
static int wl1(int F, int J, const double *W, const double *x, double *out) {
    return orc_starlet_prior(F, J, 1.0, W, x, out, NULL);
}

/* Estimate of lambda_pts from a model (App. C):
 *   lambda_pts = lambda (|| W o Phi^T fbar ||_1 - || W o Phi^T h ||_1) / sum_k <a_k> || W o Phi^T r_k ||_1,
 * fbar = (1/E) sum_i f_i the mean of the epochs' fine images f_i = h + sum_k a_ki r_k(c_k + delta_i)
 * (Eq. 9), r_k in the denominator the unit Gaussian at c_k.  The printed formula also multiplies
 * the second norm by lambda, which leaves the difference without a consistent unit; it is read
 * without that factor.  A zero denominator (no point-source flux) gives 0. */
int orc_lambda_pts_estimate(int E, int N, int f, int M, int J, double lam, const double *W, const double *params,
                            double *out) {
    if (E <= 0 || N <= 0 || f <= 0 || M < 0) return ORC_ERR_SHAPE;
    const int F = f * N;
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t oh, oa, oc, od, og, tot;
    deconv_offsets(E, N, f, M, &oh, &oa, &oc, &od, &og, &tot);
    const size_t n = (size_t)F * F;
    double *fbar = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n), *zero = calloc(2, sizeof(double));
    if (!fbar || !r || !zero) { free(fbar); free(r); free(zero); return ORC_ERR_OOM; }
    memcpy(fbar, params + oh, sizeof(double) * n);
    for (int i = 0; i < E; ++i)
        for (int k = 0; k < M; ++k) {
            double ux, uy;
            source_centre(F, f, params + oc, params + od, k, i, &ux, &uy);
            orc_add_gaussian(F, params[oa + (size_t)i * M + k] / E, ux, uy, fbar);
        }
    double l1_f = 0.0, l1_h = 0.0, den = 0.0;
    int rc = wl1(F, J, W, fbar, &l1_f);
    if (!rc) rc = wl1(F, J, W, params + oh, &l1_h);
    for (int k = 0; k < M && !rc; ++k) {
        double abar = 0.0, l1_r = 0.0, ux, uy;
        for (int i = 0; i < E; ++i) abar += params[oa + (size_t)i * M + k];
        abar /= E;
        memset(r, 0, sizeof(double) * n);
        source_centre(F, f, params + oc, zero, k, 0, &ux, &uy);
        orc_add_gaussian(F, 1.0, ux, uy, r);
        rc = wl1(F, J, W, r, &l1_r);
        den += abar * l1_r;
    }
    if (!rc) *out = den != 0.0 ? lam * (l1_f - l1_h) / den : 0.0;
    free(fbar); free(r); free(zero);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* PSF reconstruction: Eq. 2 (Moffat + pixel grid), Eq. 3, Eq. 4, Eq. 7      */
/* ------------------------------------------------------------------------- */

/* Isotropic unit-flux Moffat on the F x F fine grid centred on pixel (F/2, F/2):
 * m = (beta-1)/(pi alpha^2) (1 + rho^2/alpha^2)^(-beta); with its derivatives. */
int orc_moffat(int F, double alpha, double beta, double *m, double *dm_dalpha, double *dm_dbeta) {
    if (F <= 0 || !(alpha > 0) || !(beta > 1)) return ORC_ERR_ARG;
    int cen = F / 2;
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double rho2 = (double)(ux - cen) * (ux - cen) + (double)(uy - cen) * (uy - cen);
            double B = 1.0 + rho2 / (alpha * alpha);
            double v = (beta - 1.0) / (M_PI * alpha * alpha) * pow(B, -beta);
            size_t k = (size_t)uy * F + ux;
            m[k] = v;
            if (dm_dalpha) dm_dalpha[k] = v * (-2.0 / alpha + 2.0 * beta * rho2 / (alpha * alpha * alpha * B));
            if (dm_dbeta) dm_dbeta[k] = v * (1.0 / (beta - 1.0) - log(B));
        }
    return ORC_OK;
}

/* Packed parameters: [b F*F | alpha, beta | a S | c S*2]  (S stars). */
size_t orc_psf_param_count(int S, int N, int f) {
    size_t F = (size_t)f * N;
    return F * F + 2 + (size_t)S + (size_t)S * 2;
}

/* out[u] = sum_v s[v] g(u - v - shift): the narrow PSF convolved with the
 * Gaussian r_k of Eq. 3 displaced by (sx, sy).  The 2-D Gaussian factorises
 * exactly into 1-D factors, so the sum is taken over v_x, then over v_y. */
static void star_blur(int F, const double *s, double sx, double sy, double *tmp, double *out) {
    for (int vy = 0; vy < F; ++vy)
        for (int ux = 0; ux < F; ++ux) {
            double acc = 0.0;
            for (int vx = 0; vx < F; ++vx) acc += s[vy * F + vx] * gauss1(ux - vx - sx);
            tmp[vy * F + ux] = acc;
        }
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double acc = 0.0;
            for (int vy = 0; vy < F; ++vy) acc += tmp[vy * F + ux] * gauss1(uy - vy - sy);
            out[uy * F + ux] = acc;
        }
}

/* Literal transpose of star_blur (scatter of each term). */
static void star_blur_adjoint(int F, const double *y, double sx, double sy, double *tmp, double *out) {
    memset(tmp, 0, sizeof(double) * (size_t)F * F);
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux)
            for (int vy = 0; vy < F; ++vy) tmp[vy * F + ux] += y[uy * F + ux] * gauss1(uy - vy - sy);
    memset(out, 0, sizeof(double) * (size_t)F * F);
    for (int vy = 0; vy < F; ++vy)
        for (int ux = 0; ux < F; ++ux)
            for (int vx = 0; vx < F; ++vx) out[vy * F + vx] += tmp[vy * F + ux] * gauss1(ux - vx - sx);
}

/* Derivative of star_blur with respect to the shift: d out / d sx and d sy.
 * d/dsx g1(ux - vx - sx) = g1(.) (ux - vx - sx) / sigma^2. */
static void star_blur_dshift(int F, const double *s, double sx, double sy, double *tmp, double *tmpd, double *dx,
                             double *dy) {
    double s2 = gauss_sigma() * gauss_sigma();
    for (int vy = 0; vy < F; ++vy)
        for (int ux = 0; ux < F; ++ux) {
            double acc = 0.0, accd = 0.0;
            for (int vx = 0; vx < F; ++vx) {
                double t = ux - vx - sx;
                double g = gauss1(t);
                acc += s[vy * F + vx] * g;
                accd += s[vy * F + vx] * g * t / s2;
            }
            tmp[vy * F + ux] = acc;
            tmpd[vy * F + ux] = accd;
        }
    for (int uy = 0; uy < F; ++uy)
        for (int ux = 0; ux < F; ++ux) {
            double ax = 0.0, ay = 0.0;
            for (int vy = 0; vy < F; ++vy) {
                double t = uy - vy - sy;
                double g = gauss1(t);
                ax += tmpd[vy * F + ux] * g;
                ay += tmp[vy * F + ux] * g * t / s2;
            }
            dx[uy * F + ux] = ax;
            dy[uy * F + ux] = ay;
        }
}

/* Narrow PSF s = m(alpha, beta) + b (Eq. 2). */
static int psf_narrow(int F, const double *params, double *s, double *dma, double *dmb) {
    size_t n = (size_t)F * F;
    int rc = orc_moffat(F, params[n], params[n + 1], s, dma, dmb);
    if (rc) return rc;
    for (size_t k = 0; k < n; ++k) s[k] += params[k];
    return ORC_OK;
}

/* Shift of star k's Gaussian relative to the PSF centre pixel F/2. */
static void star_shift(int F, int f, const double *c, int k, double *sx, double *sy) {
    double u0 = 0.5 * (F - 1);
    *sx = u0 + f * c[2 * k + 0] - F / 2;
    *sy = u0 + f * c[2 * k + 1] - F / 2;
}

/* Model stamps t_k = D(a_k * (s * r_k)) on the data grid (Eq. 3, no noise). */
int orc_psf_model(int S, int N, int f, const double *params, double *model_out) {
    int F = f * N;
    size_t n = (size_t)F * F;
    double *s = malloc(sizeof(double) * n);
    if (!s) return ORC_ERR_OOM;
    int rc = psf_narrow(F, params, s, NULL, NULL);
    if (rc) { free(s); return rc; }
    const double *a = params + n + 2, *c = params + n + 2 + S;
    int err = 0;
#pragma omp parallel
    {
        double *tmp = malloc(sizeof(double) * n), *blur = malloc(sizeof(double) * n);
        if (!tmp || !blur) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(static)
            for (int k = 0; k < S; ++k) {
                double sx, sy;
                star_shift(F, f, c, k, &sx, &sy);
                star_blur(F, s, sx, sy, tmp, blur);
                for (size_t u = 0; u < n; ++u) blur[u] *= a[k];
                orc_downsample(N, f, blur, model_out + (size_t)k * N * N);
            }
        }
        free(tmp); free(blur);
    }
    free(s);
    return err ? ORC_ERR_OOM : ORC_OK;
}

/* Loss (Eq. 7) and gradient of the PSF reconstruction. parts = {chi^2, prior on b}. */
static int psf_loss_grad(int S, int N, int f, int J, double lam, const double *t, const double *sigma, const double *W,
                         const double *Wmap, const double *params, double *parts, double *grad, int nthreads) {
    if (S <= 0 || N <= 0 || f <= 0) return ORC_ERR_SHAPE;
    int F = f * N;
    if (!orc_starlet_valid(F, J)) return ORC_ERR_SHAPE;
    size_t n = (size_t)F * F;
    size_t tot = orc_psf_param_count(S, N, f);
    int nt = orc_threads(nthreads);
    double *s = malloc(sizeof(double) * n), *dma = malloc(sizeof(double) * n), *dmb = malloc(sizeof(double) * n);
    double *chi = calloc((size_t)S, sizeof(double));
    double *gs_star = grad ? calloc(n * (size_t)S, sizeof(double)) : NULL;
    if (!s || !dma || !dmb || !chi || (grad && !gs_star)) {
        free(s); free(dma); free(dmb); free(chi); free(gs_star);
        return ORC_ERR_OOM;
    }
    int rc = psf_narrow(F, params, s, dma, dmb);
    if (rc) { free(s); free(dma); free(dmb); free(chi); free(gs_star); return rc; }
    if (grad) memset(grad, 0, sizeof(double) * tot);
    const double *a = params + n + 2, *c = params + n + 2 + S;
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        double *tmp = malloc(sizeof(double) * n), *tmpd = malloc(sizeof(double) * n);
        double *blur = malloc(sizeof(double) * n), *ey = malloc(sizeof(double) * n);
        double *dx = malloc(sizeof(double) * n), *dy = malloc(sizeof(double) * n);
        double *model = malloc(sizeof(double) * (size_t)N * N), *e = malloc(sizeof(double) * (size_t)N * N);
        if (!tmp || !tmpd || !blur || !ey || !dx || !dy || !model || !e) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int k = 0; k < S; ++k) {
                double sx, sy;
                star_shift(F, f, c, k, &sx, &sy);
                star_blur(F, s, sx, sy, tmp, blur);
                for (size_t u = 0; u < n; ++u) ey[u] = a[k] * blur[u];
                orc_downsample(N, f, ey, model);
                double c2 = 0.0;
                for (int p = 0; p < N * N; ++p) {
                    size_t ip = (size_t)k * N * N + p;
                    double w = inv_var(sigma[ip]);
                    double r = t[ip] - model[p];
                    c2 += 0.5 * w * r * r;
                    e[p] = -w * r;
                }
                chi[k] = c2;
                if (!grad) continue;
                orc_downsample_adjoint(N, f, e, ey);
                /* d/da_k = <D^T e, s * r_k> */
                double ga = 0.0;
                for (size_t u = 0; u < n; ++u) ga += ey[u] * blur[u];
                grad[n + 2 + k] = ga;
                /* d/dc_k = f a_k <D^T e, d(s * r_k)/d shift> */
                star_blur_dshift(F, s, sx, sy, tmp, tmpd, dx, dy);
                double gx = 0.0, gy = 0.0;
                for (size_t u = 0; u < n; ++u) { gx += ey[u] * dx[u]; gy += ey[u] * dy[u]; }
                grad[n + 2 + S + 2 * k + 0] = f * a[k] * gx;
                grad[n + 2 + S + 2 * k + 1] = f * a[k] * gy;
                /* d/ds from this star: a_k B_k^T D^T e */
                double *gsk = gs_star + (size_t)k * n;
                star_blur_adjoint(F, ey, sx, sy, tmp, gsk);
                for (size_t u = 0; u < n; ++u) gsk[u] *= a[k];
            }
        }
        free(tmp); free(tmpd); free(blur); free(ey); free(dx); free(dy); free(model); free(e);
    }
    if (err) { free(s); free(dma); free(dmb); free(chi); free(gs_star); return ORC_ERR_OOM; }
    double chi2 = 0.0;
    for (int k = 0; k < S; ++k) chi2 += chi[k];
    double prior = 0.0;
    double *gprior = grad ? malloc(sizeof(double) * n) : NULL;
    rc = prior_w(F, J, lam, W, Wmap, params, &prior, gprior);
    if (grad && rc == ORC_OK) {
        double galpha = 0.0, gbeta = 0.0;
        for (size_t u = 0; u < n; ++u) {
            double gs = 0.0;
            for (int k = 0; k < S; ++k) gs += gs_star[(size_t)k * n + u];
            grad[u] = gs + gprior[u]; /* s = m + b: ds/db = 1 */
            galpha += gs * dma[u];
            gbeta += gs * dmb[u];
        }
        grad[n] = galpha;
        grad[n + 1] = gbeta;
    }
    parts[0] = chi2;
    parts[1] = prior;
    free(gprior); free(s); free(dma); free(dmb); free(chi); free(gs_star);
    return rc;
}

int orc_psf_loss_grad(int S, int N, int f, int J, double lam, const double *t, const double *sigma, const double *W,
                      const double *params, double *parts, double *grad, int nthreads) {
    return psf_loss_grad(S, N, f, J, lam, t, sigma, W, NULL, params, parts, grad, nthreads);
}

/* The PSF loss with the per-coefficient prior weights Wmap [J-1][F][F]. */
int orc_psf_loss_grad_map(int S, int N, int f, int J, double lam, const double *t, const double *sigma,
                          const double *Wmap, const double *params, double *parts, double *grad, int nthreads) {
    return psf_loss_grad(S, N, f, J, lam, t, sigma, NULL, Wmap, params, parts, grad, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Optimiser: AdaBelief (Zhuang et al. 2020, the published update) and Adam, */
/* followed by projection onto per-element lower bounds.  Used as in sec. 2.4 */
/* ------------------------------------------------------------------------- */

/* kind 0 = AdaBelief, 1 = Adam.  t is the 1-based step index of this update.
 * lo[k] = -inf for unconstrained elements.  hi[k] = +inf likewise. */
int orc_optim_step(int kind, long n, double *theta, const double *g, double *m, double *v, long t, const double *lr,
                   double beta1, double beta2, double eps, const double *lo, const double *hi) {
    if (n < 0 || t < 1) return ORC_ERR_ARG;
    double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
    for (long k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        if (kind == 0) {
            double dev = g[k] - m[k];
            v[k] = beta2 * v[k] + (1.0 - beta2) * dev * dev + eps;
        } else {
            v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        }
        double mh = m[k] / bc1, vh = v[k] / bc2;
        double th = theta[k] - lr[k] * mh / (sqrt(vh) + eps);
        if (th < lo[k]) th = lo[k];
        if (th > hi[k]) th = hi[k];
        theta[k] = th;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Noise propagation to the starlet coefficients (sec. 2.3, App. B).          */
/* ------------------------------------------------------------------------- */

/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers:
 * as easy as 1, 2, 3"): ten rounds of two 64 x 64 -> 128-bit products on a
 * four-word counter, the two-word key bumped by the Weyl constants between
 * rounds.  One block: counter ctr, key key -> four 64-bit words. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normal number n of stream `seed`: block b = n / 4 of Philox4x64-10
 * with counter (b, 0, 0, 0) and key (seed, 0); words (0, 1) and (2, 3) give
 * two Box-Muller pairs from the uniforms u = ((w >> 40) + 1) 2^-24 in (0, 1]:
 * z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b) for n mod 4 = (0, 1) and
 * (2, 3).  (24-bit uniforms: every single-precision implementation of the
 * same stream draws the same u exactly.) */
double orc_normal(uint64_t seed, uint64_t n) {
    const uint64_t ctr[4] = {n >> 2, 0, 0, 0}, key[2] = {seed, 0};
    uint64_t w[4];
    orc_philox4x64(ctr, key, w);
    const int q = (int)(n & 3), pair = q >> 1;
    const double ua = (double)((w[2 * pair] >> 40) + 1) * 0x1p-24;
    const double ub = (double)((w[2 * pair + 1] >> 40) + 1) * 0x1p-24;
    const double r = sqrt(-2.0 * log(ua));
    return (q & 1) ? r * sin(2.0 * M_PI * ub) : r * cos(2.0 * M_PI * ub);
}

/* Starlet weights by Monte Carlo noise propagation (sec. 2.3): realisation r
 * draws z_r on the fine grid (normal number r F^2 + u of the stream `seed`),
 * forms (C^)^-1 dd = z / sigma^ with sigma^ the effective noise of the
 * co-added epochs, sigma_eff(p)^-2 = sum_i sigma_i(p)^-2, replicated onto the
 * f x f fine pixels of data pixel p (sigma = +inf masks a pixel), propagates it
 * with S_1^T (the correlation with epoch 1's narrow PSF) and the starlet
 * analysis.  Outputs, for each detail plane w_{j+1}, j = 0..J-2:
 *   W_map [J-1][F][F]: the sample standard deviation (n - 1) over the n_real
 *                      realisations of each coefficient;
 *   W_scale [J-1]:     the sample standard deviation (n F^2 - 1) of all the
 *                      plane's coefficients of all realisations, the one number
 *                      per scale the prior of Eq. 6 takes.
 * Either output may be NULL. */
int orc_noise_weights(int N, int f, int K, int J, int E, const double *sigma, const double *s1, int n_real,
                      uint64_t seed, double *W_map, double *W_scale) {
    const int F = f * N;
    if (N < 1 || f < 1 || K < 1 || !orc_starlet_valid(F, J) || n_real < 2 || E < 1) return ORC_ERR_SHAPE;
    const size_t n = (size_t)F * F, nd = (size_t)(J - 1) * n;
    /* realisations split into contiguous per-thread ranges with private sums, added in thread order */
    int nt = omp_in_parallel() ? 1 : omp_get_max_threads();
    if (nt > n_real) nt = n_real;
    double *isig = malloc(sizeof(double) * n), *work = malloc(sizeof(double) * (size_t)nt * (2 + J) * n);
    double *part1 = calloc((size_t)nt * nd, sizeof(double)), *part2 = calloc((size_t)nt * nd, sizeof(double));
    double *s1sum = calloc(nd, sizeof(double)), *s2sum = calloc(nd, sizeof(double));
    if (!isig || !work || !part1 || !part2 || !s1sum || !s2sum) {
        free(isig); free(work); free(part1); free(part2); free(s1sum); free(s2sum);
        return ORC_ERR_OOM;
    }
    for (int p = 0; p < N * N; ++p) {
        double iv = 0.0;
        for (int i = 0; i < E; ++i) {
            const double sg = sigma[(size_t)i * N * N + p];
            if (isfinite(sg)) iv += 1.0 / (sg * sg);
        }
        const double v = sqrt(iv);  /* 1 / sigma_eff */
        const int py = p / N, px = p % N;
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) isig[(size_t)(f * py + a) * F + (f * px + b)] = v;
    }
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        double *x = work + (size_t)t * (2 + J) * n, *y = x + n, *planes = y + n;
        double *p1 = part1 + (size_t)t * nd, *p2 = part2 + (size_t)t * nd;
        const int r0 = (int)((long)n_real * t / T), r1 = (int)((long)n_real * (t + 1) / T);
        for (int r = r0; r < r1; ++r) {
            for (size_t u = 0; u < n; ++u) x[u] = orc_normal(seed, (uint64_t)r * n + u) * isig[u];
            orc_conv_same_adjoint(F, K, x, s1, y);
            orc_starlet_analysis(F, J, y, planes);
            for (size_t k = 0; k < nd; ++k) {
                p1[k] += planes[k];
                p2[k] += planes[k] * planes[k];
            }
        }
    }
    for (int t = 0; t < nt; ++t)
        for (size_t k = 0; k < nd; ++k) {
            s1sum[k] += part1[(size_t)t * nd + k];
            s2sum[k] += part2[(size_t)t * nd + k];
        }
    for (int j = 0; j < J - 1; ++j) {
        double t1 = 0.0, t2 = 0.0;
        for (size_t u = 0; u < n; ++u) {
            const size_t k = (size_t)j * n + u;
            t1 += s1sum[k];
            t2 += s2sum[k];
            if (W_map) {
                const double mean = s1sum[k] / n_real;
                const double var = (s2sum[k] - n_real * mean * mean) / (n_real - 1);
                W_map[k] = sqrt(var > 0.0 ? var : 0.0);
            }
        }
        if (W_scale) {
            const double m = (double)n_real * (double)n, mean = t1 / m, var = (t2 - m * mean * mean) / (m - 1.0);
            W_scale[j] = sqrt(var > 0.0 ? var : 0.0);
        }
    }
    free(isig); free(work); free(part1); free(part2); free(s1sum); free(s2sum);
    return ORC_OK;
}
