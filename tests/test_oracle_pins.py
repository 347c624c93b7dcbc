"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one oracle function to a closed form, a library routine for a
special case, an exact identity, a published table, or finite differences, so
that a dropped term, a wrong sign or index, or a transposed operand fails here.
"""
import numpy as np
import pytest
import scipy.fft
import scipy.ndimage
import scipy.signal

import oracle
from paper_2402_08725_gb300 import synthetic as syn

B3 = np.array([1, 4, 6, 4, 1], dtype=np.float64) / 16.0
RNG = np.random.default_rng(12345)


# --- S: narrow-PSF convolution (Eq. 8, Eq. 10) -------------------------------------

@pytest.mark.parametrize("F,K", [(12, 5), (12, 4), (9, 13), (16, 16)])
def test_conv_same_matches_scipy_full_crop(F, K):
    """S is the 'full' linear convolution cropped at the kernel origin K//2."""
    x, s = RNG.standard_normal((F, F)), RNG.standard_normal((K, K))
    o = K // 2
    ref = scipy.signal.convolve2d(x, s, mode="full")[o:o + F, o:o + F]
    np.testing.assert_allclose(oracle.conv_same(x, s), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("F,K", [(16, 7), (16, 8)])
def test_conv_same_matches_fft_product(F, K):
    """Zero-padded FFT product (pad >= F + K - 1) gives the same linear convolution."""
    x, s = RNG.standard_normal((F, F)), RNG.standard_normal((K, K))
    P = F + K - 1
    full = np.real(scipy.fft.ifft2(scipy.fft.fft2(x, (P, P)) * scipy.fft.fft2(s, (P, P))))
    o = K // 2
    np.testing.assert_allclose(oracle.conv_same(x, s), full[o:o + F, o:o + F], atol=1e-10)


@pytest.mark.parametrize("K", [5, 6, 64])
def test_delta_psf_is_identity(K):
    F = 20
    x = RNG.standard_normal((F, F))
    s = np.zeros((K, K))
    s[K // 2, K // 2] = 1.0
    np.testing.assert_array_equal(oracle.conv_same(x, s), x)


def test_asymmetric_kernel_orientation():
    """A kernel with a single tap at q = o + (0, 1) moves an image one column right (true convolution)."""
    F, K = 10, 5
    x = RNG.standard_normal((F, F))
    s = np.zeros((K, K))
    s[K // 2, K // 2 + 1] = 1.0
    out = oracle.conv_same(x, s)
    np.testing.assert_array_equal(out[:, 1:], x[:, :-1])
    np.testing.assert_array_equal(out[:, 0], 0.0)


@pytest.mark.parametrize("F,K", [(14, 5), (14, 6), (8, 13)])
def test_conv_adjoint_dot_product(F, K):
    x, y, s = RNG.standard_normal((F, F)), RNG.standard_normal((F, F)), RNG.standard_normal((K, K))
    lhs = np.vdot(oracle.conv_same(x, s), y)
    rhs = np.vdot(x, oracle.conv_same_adjoint(y, s))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


# --- D: block-sum downsampling ----------------------------------------------------

@pytest.mark.parametrize("N,f", [(8, 2), (5, 3), (4, 1)])
def test_downsample_flux_and_adjoint(N, f):
    x = RNG.standard_normal((N * f, N * f))
    dx = oracle.downsample(x, f)
    assert abs(dx.sum() - x.sum()) <= 1e-12 * np.abs(x).sum()
    # a library special case: block sum = reshape-sum
    np.testing.assert_allclose(dx, x.reshape(N, f, N, f).sum(axis=(1, 3)), atol=1e-13)
    e = RNG.standard_normal((N, N))
    lhs, rhs = np.vdot(dx, e), np.vdot(x, oracle.downsample_adjoint(e, f))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


# --- starlet transform (Eq. 6) -----------------------------------------------------

@pytest.mark.parametrize("F,J", [(16, 3), (33, 4), (64, 6)])
def test_starlet_exact_reconstruction(F, J):
    h = RNG.standard_normal((F, F)) * 100
    planes = oracle.starlet_analysis(h, J)
    rec = planes.sum(axis=0)
    assert np.max(np.abs(rec - h)) <= 1e-12 * np.max(np.abs(h))


def test_starlet_constant_image_has_no_detail():
    planes = oracle.starlet_analysis(np.full((20, 20), 3.7), 4)
    assert np.max(np.abs(planes[:-1])) < 1e-13
    np.testing.assert_allclose(planes[-1], 3.7, atol=1e-13)


def _dilated(j):
    k = np.zeros(4 * (1 << j) + 1)
    k[:: 1 << j] = B3
    return k


def test_starlet_smoothing_matches_scipy_mirror_mode():
    """One level of the transform = separable correlation with the dilated B3
    filter under whole-sample mirror borders (scipy mode 'mirror')."""
    F, J = 23, 4
    h = RNG.standard_normal((F, F))
    planes = oracle.starlet_analysis(h, J)
    c = h.copy()
    for j in range(J - 1):
        k = _dilated(j)
        cn = scipy.ndimage.correlate1d(c, k, axis=1, mode="mirror")
        cn = scipy.ndimage.correlate1d(cn, k, axis=0, mode="mirror")
        np.testing.assert_allclose(planes[j], c - cn, atol=1e-12)
        c = cn
    np.testing.assert_allclose(planes[-1], c, atol=1e-12)


def test_starlet_delta_atoms_closed_form():
    """Coarse planes of a centred delta are outer products of the 1-D cascade of
    dilated B3 filters (closed form, no border contact)."""
    F, J = 65, 4
    h = np.zeros((F, F))
    h[32, 32] = 1.0
    planes = oracle.starlet_analysis(h, J)
    casc = np.array([1.0])
    coarse = [h]
    for j in range(J - 1):
        casc = np.convolve(casc, _dilated(j))
        img = np.zeros((F, F))
        r = len(casc) // 2
        img[32 - r:32 + r + 1, 32 - r:32 + r + 1] = np.outer(casc, casc)
        coarse.append(img)
    for j in range(J - 1):
        np.testing.assert_allclose(planes[j], coarse[j] - coarse[j + 1], atol=1e-15)
    np.testing.assert_allclose(planes[-1], coarse[-1], atol=1e-15)


def test_starlet_white_noise_levels_match_published_table():
    """Per-scale std of the starlet of unit white noise matches the published
    B3-starlet values 0.8908, 0.2007, 0.0856, 0.0413 (Starck & Murtagh)."""
    rng = np.random.default_rng(7)
    h = rng.standard_normal((256, 256))
    planes = oracle.starlet_analysis(h, 5)
    inner = planes[:, 32:-32, 32:-32]
    got = inner[:4].std(axis=(1, 2))
    np.testing.assert_allclose(got, [0.8908, 0.2007, 0.0856, 0.0413], rtol=0.05)


@pytest.mark.parametrize("F,J", [(16, 3), (24, 4), (64, 6)])
def test_starlet_adjoint_dot_product(F, J):
    x = RNG.standard_normal((F, F))
    y = RNG.standard_normal((J, F, F))
    lhs = np.vdot(oracle.starlet_analysis(x, J), y)
    rhs = np.vdot(x, oracle.starlet_adjoint(y))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_starlet_prior_value_and_subgradient():
    F, J, lam = 24, 4, 2.5
    W = np.array([1.3, 0.4, 0.2])
    h = RNG.standard_normal((F, F)) * 10
    planes = oracle.starlet_analysis(h, J)
    want = lam * sum(W[j] * np.abs(planes[j]).sum() for j in range(J - 1))
    p, g = oracle.starlet_prior(h, J, lam, W)
    assert abs(p - want) <= 1e-12 * want
    # gradient = adjoint of the sign pattern (coarse plane unpenalised)
    y = np.concatenate([lam * W[:, None, None] * np.sign(planes[:-1]), np.zeros((1, F, F))])
    np.testing.assert_allclose(g, oracle.starlet_adjoint(y), atol=1e-12)
    # central differences away from kinks
    step = 1e-6
    for _ in range(6):
        u = tuple(RNG.integers(0, F, size=2))
        hp, hm = h.copy(), h.copy()
        hp[u] += step
        hm[u] -= step
        fd = (oracle.starlet_prior(hp, J, lam, W, grad=False) - oracle.starlet_prior(hm, J, lam, W, grad=False)) / (
            2 * step)
        assert abs(fd - g[u]) <= 1e-6 * max(1.0, abs(g[u]))


# --- narrow Gaussian r (Eq. 1: FWHM 2 fine px) --------------------------------------

def test_gaussian_half_maximum_at_one_pixel():
    F = 21
    img = oracle.add_gaussian(np.zeros((F, F)), 1.0, 10.0, 10.0)
    # FWHM = 2 px: the value one pixel from the centre is half the peak
    assert abs(img[10, 11] / img[10, 10] - 0.5) < 1e-14
    assert abs(img[11, 10] / img[10, 10] - 0.5) < 1e-14
    # analytic unit-flux normalisation of the peak: 1 / (2 pi sigma^2) = ln 2 / pi
    assert abs(img[10, 10] - np.log(2) / np.pi) < 1e-15


@pytest.mark.parametrize("x0", [0.0, 0.25, 0.5])
def test_gaussian_sampled_sum_poisson_bound(x0):
    """Sum of the point-sampled unit Gaussian equals its Poisson series
    (1 + 2 sum_k exp(-2 pi^2 sigma^2 k^2) cos(2 pi k x0)) per axis."""
    F = 41
    img = oracle.add_gaussian(np.zeros((F, F)), 1.0, 20.0 + x0, 20.0 + x0)
    sig2 = 1.0 / (2 * np.log(2))
    ks = np.arange(1, 6)
    axis = 1 + 2 * np.sum(np.exp(-2 * np.pi ** 2 * sig2 * ks ** 2) * np.cos(2 * np.pi * ks * x0))
    assert abs(img.sum() - axis ** 2) < 1e-13
    assert abs(img.sum() - 1) < 2.7e-6


# --- Moffat (Eq. 2) ------------------------------------------------------------------

def test_moffat_flux_half_max_and_derivatives():
    # flux 1 up to the tail outside the grid, (1 + R^2/alpha^2)^(1-beta) for the
    # inscribed disc; alpha wide enough that point sampling does not alias
    F, wide = 401, 6.0
    m, _, _ = oracle.moffat(F, wide, 3.0)
    R = F // 2
    tail = (1 + R * R / wide ** 2) ** (1 - 3.0)
    assert -1e-12 < 1.0 - m.sum() < tail + 1e-12
    alpha, beta = 2.0, 3.0
    fwhm = 2 * alpha * np.sqrt(2 ** (1 / beta) - 1)
    m_small, _, _ = oracle.moffat(65, alpha, beta)
    peak = (beta - 1) / (np.pi * alpha ** 2)
    assert abs(m_small[32, 32] - peak) < 1e-15
    # half maximum at radius FWHM/2 (closed form of the profile)
    rho = fwhm / 2
    assert abs((1 + rho ** 2 / alpha ** 2) ** (-beta) - 0.5) < 1e-14
    for h_a, h_b in [(1e-6, 0), (0, 1e-6)]:
        mp, _, _ = oracle.moffat(33, alpha + h_a, beta + h_b)
        mm, _, _ = oracle.moffat(33, alpha - h_a, beta - h_b)
        fd = (mp - mm) / 2e-6
        _, da33, db33 = oracle.moffat(33, alpha, beta)
        ref = da33 if h_a else db33
        np.testing.assert_allclose(fd, ref, rtol=1e-6, atol=1e-10)


# --- full losses: finite differences -----------------------------------------------

def _kink_margin(planes):
    return float(np.min(np.abs(planes[:-1])))


def _fd_check(fun, params, idx, steps, rtol, atol_floor):
    """Central differences; the tolerance adds the cancellation noise |L| eps / h."""
    L0, g = fun(params)
    for k in idx:
        h = steps[k]
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd = (fun(pp, grad=False)[0] - fun(pm, grad=False)[0]) / (2 * h)
        noise = 20 * abs(L0) * np.finfo(float).eps / h
        assert abs(fd - g[k]) <= rtol * max(abs(g[k]), atol_floor) + noise, (k, fd, g[k])


def _steps(params, n_img, margin, rel=1e-6):
    """Relative steps, but image pixels move by less than the smallest starlet
    coefficient so that no |.| of the prior changes sign (sign(0) = 0 reading)."""
    st = rel * np.maximum(1.0, np.abs(params))
    st[:n_img] = np.minimum(st[:n_img], 0.1 * margin)
    return st


@pytest.mark.parametrize("lam", [0.0, 0.7])
def test_deconv_gradient_central_differences(lam):
    fd_ = syn.small_deconv(seed=3, E=3, N=12, f=2, K=9, M=2, J=3, lam=lam)
    P = fd_.params.astype(np.float64)
    F = fd_.F
    margin = _kink_margin(oracle.starlet_analysis(P[:F * F].reshape(F, F), fd_.J))
    assert margin > 1e-9

    def fun(p, grad=True):
        L, _, g, _ = oracle.deconv_loss_grad(fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, lam, fd_.d,
                                             fd_.sigma, fd_.s, fd_.W, p, grad=grad)
        return L, g

    rng = np.random.default_rng(0)
    idx = list(rng.choice(F * F, 12, replace=False)) + list(range(F * F, P.size))
    _fd_check(fun, P, idx, _steps(P, F * F, margin), 1e-6, 1e-3)


@pytest.mark.parametrize("lam", [0.0, 0.5])
def test_psf_gradient_central_differences(lam):
    pb = syn.small_psf(seed=5, S=2, N=10, f=2, J=3, lam=lam)
    P = pb.params.astype(np.float64)
    F = pb.F
    margin = _kink_margin(oracle.starlet_analysis(P[:F * F].reshape(F, F), pb.J))
    assert margin > 1e-12

    def fun(p, grad=True):
        L, _, g = oracle.psf_loss_grad(pb.S, pb.N, pb.f, pb.J, lam, pb.t, pb.sigma, pb.W, p, grad=grad)
        return L, g

    rng = np.random.default_rng(1)
    idx = list(rng.choice(F * F, 12, replace=False)) + list(range(F * F, P.size))
    _fd_check(fun, P, idx, _steps(P, F * F, margin), 1e-6, 1e-3)


# --- model invariants --------------------------------------------------------------

def _single_source_params(E, N, f, M, c, amp):
    F = f * N
    return syn.pack_deconv(np.zeros((F, F)), np.full((E, M), amp), np.asarray(c, float).reshape(M, 2),
                           np.zeros((E, 2)), np.zeros(E)).astype(np.float64)


def test_point_source_centroid_convention():
    """A source at offset c (data px from the stamp centre (N-1)/2) has its
    model centroid at (N-1)/2 + c, x along columns.  The input PSF is a wide
    Gaussian (sigma 3 fine px, cut at 6.7 sigma) so that the block sum does not
    alias the centroid (aliasing ~ exp(-2 pi^2 sigma_tot^2 / f^2) < 1e-20)."""
    E, N, f, K, M = 1, 40, 2, 41, 1
    yy, xx = np.mgrid[0:K, 0:K] - K // 2
    s = np.exp(-(xx ** 2 + yy ** 2) / (2 * 3.0 ** 2))[None]
    s /= s.sum()
    for c in [(0.0, 0.0), (1.25, 0.0), (0.0, -2.5), (1.0, 0.75)]:
        P = _single_source_params(E, N, f, M, c, 1000.0)
        mod = oracle.deconv_model(E, N, f, K, M, s, P)[0]
        y, x = np.mgrid[0:N, 0:N]
        cx, cy = (mod * x).sum() / mod.sum(), (mod * y).sum() / mod.sum()
        assert abs(cx - ((N - 1) / 2 + c[0])) < 1e-5
        assert abs(cy - ((N - 1) / 2 + c[1])) < 1e-5
        assert abs(mod.sum() - 1000.0) < 1e-2   # flux conserved by S (sum 1) and D


def test_integer_shift_moves_model_by_one_data_pixel():
    E, N, f, K, M = 1, 20, 2, 7, 1
    s = syn.moffat_stack(K, [2.0], [2.5]).astype(np.float64)
    m0 = oracle.deconv_model(E, N, f, K, M, s, _single_source_params(E, N, f, M, (0.0, 0.0), 500.0))[0]
    m1 = oracle.deconv_model(E, N, f, K, M, s, _single_source_params(E, N, f, M, (1.0, 0.0), 500.0))[0]
    np.testing.assert_allclose(m1[:, 1:], m0[:, :-1], atol=1e-9)


def test_background_gamma_adds_f2_per_data_pixel():
    E, N, f, K, M = 2, 8, 3, 5, 1
    s = syn.moffat_stack(K, [2.0, 2.0], [2.5, 2.5]).astype(np.float64)
    P = _single_source_params(E, N, f, M, (0.0, 0.0), 10.0)
    m0 = oracle.deconv_model(E, N, f, K, M, s, P)
    P[-E:] = [0.5, -1.0]
    m1 = oracle.deconv_model(E, N, f, K, M, s, P)
    np.testing.assert_allclose(m1 - m0, np.array([0.5, -1.0])[:, None, None] * f * f + 0 * m0, atol=1e-12)


def test_noiseless_truth_zero_loss_and_noisy_chi2_statistics():
    fd_ = syn.small_deconv(seed=11, E=4, N=16, f=2, K=11, M=2, J=3, lam=0.0)
    P = fd_.params.astype(np.float64)
    model = oracle.deconv_model(fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.s, P)
    sig = np.full_like(model, 4.0)
    L, parts, g, _ = oracle.deconv_loss_grad(fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, 0.0, model, sig, fd_.s,
                                             fd_.W, P)
    assert L == 0.0 and np.all(g == 0.0)
    rng = np.random.default_rng(2)
    npix = model.size
    vals = []
    for _ in range(20):
        d = model + sig * rng.standard_normal(model.shape)
        vals.append(2 * oracle.deconv_loss_grad(fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, 0.0, d, sig, fd_.s,
                                                fd_.W, P, grad=False)[0] / npix)
    assert abs(np.mean(vals) - 1.0) < 4 * np.sqrt(2.0 / npix) / np.sqrt(20)


def test_masked_pixels_do_not_contribute():
    fd_ = syn.small_deconv(seed=12, E=2, N=10, f=2, K=7, M=1, J=3, lam=0.5)
    sig = fd_.sigma.astype(np.float64).copy()
    d2 = fd_.d.astype(np.float64).copy()
    sig[0, 3, 4] = np.inf
    d2[0, 3, 4] += 1e6
    args = (fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, fd_.lam)
    a = oracle.deconv_loss_grad(*args, fd_.d, sig, fd_.s, fd_.W, fd_.params)
    b = oracle.deconv_loss_grad(*args, d2, sig, fd_.s, fd_.W, fd_.params)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[2], b[2])


def test_epochs_add_independently():
    """The chi^2 and its gradient are sums over epochs (the multi-GPU design
    shards epochs): two halves of the epochs give the whole."""
    fd_ = syn.small_deconv(seed=13, E=4, N=12, f=2, K=7, M=2, J=3, lam=0.0)
    F = fd_.F
    full = oracle.deconv_loss_grad(fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, 0.0, fd_.d, fd_.sigma, fd_.s, fd_.W,
                                   fd_.params)
    h, a, c, dl, gm = syn.unpack_deconv(fd_.params, fd_.E, fd_.N, fd_.f, fd_.M)
    tot_h = np.zeros(F * F)
    tot_c = np.zeros(2 * fd_.M)
    L = 0.0
    for sl in (slice(0, 2), slice(2, 4)):
        P = syn.pack_deconv(h, a[sl], c, dl[sl], gm[sl])
        r = oracle.deconv_loss_grad(2, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J, 0.0, fd_.d[sl], fd_.sigma[sl], fd_.s[sl],
                                    fd_.W, P)
        L += r[0]
        tot_h += r[2][:F * F]
        tot_c += r[2][F * F + 2 * fd_.M:F * F + 4 * fd_.M]
    assert abs(L - full[0]) <= 1e-12 * full[0]
    np.testing.assert_allclose(tot_h, full[2][:F * F], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(tot_c, full[2][F * F + fd_.E * fd_.M:F * F + fd_.E * fd_.M + 2 * fd_.M], rtol=1e-10)


# --- optimiser -------------------------------------------------------------------

def _one(kind, g, lr=0.1, theta=1.0, lo=-np.inf):
    a = lambda v: np.array([v], dtype=np.float64)
    th, m, v = a(theta), a(0.0), a(0.0)
    oracle.optim_step(kind, th, a(g), m, v, 1, a(lr), 0.9, 0.999, 1e-16, a(lo), a(np.inf))
    return th[0], m[0], v[0]


def test_adabelief_and_adam_first_step_closed_forms():
    # Adam: the first bias-corrected step is lr * sign(g)
    assert abs(_one(oracle.ADAM, 2.0)[0] - 0.9) < 1e-12
    assert abs(_one(oracle.ADAM, -3.0)[0] - 1.1) < 1e-12
    # AdaBelief (published update): m1 = (1-b1) g, s1 = (1-b2)(g - m1)^2 + eps,
    # so the first step is lr * g / |b1 g| = lr / b1 * sign(g)
    th, m, v = _one(oracle.ADABELIEF, 2.0)
    assert abs(m - 0.2) < 1e-15
    assert abs(v - (0.001 * 1.8 ** 2 + 1e-16)) < 1e-14 * v
    assert abs(th - (1.0 - 0.1 / 0.9)) < 1e-12
    # projection onto the lower bound
    assert _one(oracle.ADABELIEF, 2.0, lr=5.0, lo=0.0)[0] == 0.0


def test_recovery_of_point_sources_noiseless():
    """Noiseless data made by the model: AdaBelief on (a, c) with h and delta held
    at the truth recovers amplitudes and positions."""
    fd_ = syn.small_deconv(seed=21, E=3, N=14, f=2, K=9, M=2, J=3, lam=0.0)
    E, N, f, K, M, J = fd_.E, fd_.N, fd_.f, fd_.K, fd_.M, fd_.J
    F = f * N
    truth = fd_.params.astype(np.float64)
    d = oracle.deconv_model(E, N, f, K, M, fd_.s, truth)
    sig = np.full_like(d, 3.0)
    h, a, c, dl, gm = syn.unpack_deconv(truth, E, N, f, M)
    start = syn.pack_deconv(h, a * 1.2, c + 0.3, dl, gm).astype(np.float64)
    n = start.size
    lr = np.zeros(n)
    oa, oc = F * F, F * F + E * M
    lr[oa:oc] = 0.02 * np.abs(a).mean()
    lr[oc:oc + 2 * M] = 0.01
    lo, hi = np.full(n, -np.inf), np.full(n, np.inf)
    lo[oa:oc] = 0.0
    th, m, v = start.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 1501):
        _, _, g, _ = oracle.deconv_loss_grad(E, N, f, K, M, J, 0.0, d, sig, fd_.s, fd_.W, th)
        oracle.optim_step(oracle.ADABELIEF, th, g, m, v, t, lr, 0.9, 0.999, 1e-16, lo, hi)
        if t == 1000:
            lr *= 0.1
    _, a_r, c_r, _, _ = syn.unpack_deconv(th, E, N, f, M)
    np.testing.assert_allclose(a_r, a, rtol=1e-3)
    np.testing.assert_allclose(c_r, c, atol=1e-3)
