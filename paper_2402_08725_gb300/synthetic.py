"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path (tests, benchmark) and the FP64 oracle.
It holds none of the method's arithmetic: it never rasterises the model,
convolves by a narrow PSF, downsamples, or evaluates the loss.  Scenes are
rendered directly at data resolution with simple analytic profiles, so the
data resemble what the model produces without being made by it.  Where a test
needs data made exactly by the model (noiseless recovery), the test makes them
with the oracle.

Workload shapes follow the paper's science cases, whose datasets are not
available: LSST-like lensed quasars (sec. 4.2), SN Ia host fields (sec. 4.1)
and a JWST-like wide field (sec. 4.3); PSF reconstruction from star cutouts
(sec. 3).  All values are float32; every generator takes a seed.

Packed parameter layouts (shared by the C ABI, the oracle and the tests):
  deconvolution  [h F*F | a E*M | c M*2 | delta E*2 | Gamma E]
  PSF fit        [b F*F | alpha, beta | a S | c S*2]
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2402087250

# Standard deviation of each detail plane of the B3 starlet for unit white
# noise (a published property of the transform, Starck & Murtagh); used only to
# give the synthetic prior weights W a realistic scale-to-scale ratio.
_STARLET_NOISE = np.array([0.8908, 0.2007, 0.0856, 0.0413, 0.0205, 0.0103, 0.0052, 0.0026])


@dataclass
class DeconvField:
    """One joint-deconvolution problem (one field, all its epochs)."""
    E: int
    N: int
    f: int
    K: int
    M: int
    J: int
    lam: float
    d: np.ndarray       # [E, N, N] data
    sigma: np.ndarray   # [E, N, N] noise std (inf = masked)
    s: np.ndarray       # [E, K, K] narrow PSFs, origin (K//2, K//2), sum 1
    W: np.ndarray       # [J-1] prior weight per detail scale
    params: np.ndarray  # packed evaluation point
    meta: dict = field(default_factory=dict)

    @property
    def F(self) -> int:
        return self.f * self.N

    @property
    def n_params(self) -> int:
        return self.F * self.F + self.E * self.M + 2 * self.M + 2 * self.E + self.E

    @property
    def epoch_pixels(self) -> int:
        return self.E * self.N * self.N


@dataclass
class PsfProblem:
    """PSF reconstruction from S star cutouts."""
    S: int
    N: int
    f: int
    J: int
    lam: float
    t: np.ndarray       # [S, N, N] star stamps
    sigma: np.ndarray   # [S, N, N]
    W: np.ndarray       # [J-1]
    params: np.ndarray  # packed evaluation point
    meta: dict = field(default_factory=dict)

    @property
    def F(self) -> int:
        return self.f * self.N

    @property
    def n_params(self) -> int:
        return self.F * self.F + 2 + self.S + 2 * self.S

    @property
    def epoch_pixels(self) -> int:
        return self.S * self.N * self.N


# --- layout helpers ------------------------------------------------------------

def pack_deconv(h, a, c, delta, gamma) -> np.ndarray:
    return np.concatenate([np.ravel(h), np.ravel(a), np.ravel(c), np.ravel(delta), np.ravel(gamma)]).astype(np.float32)


def unpack_deconv(p, E, N, f, M):
    F = f * N
    o = 0
    h = p[o:o + F * F].reshape(F, F); o += F * F
    a = p[o:o + E * M].reshape(E, M); o += E * M
    c = p[o:o + 2 * M].reshape(M, 2); o += 2 * M
    dl = p[o:o + 2 * E].reshape(E, 2); o += 2 * E
    g = p[o:o + E]
    return h, a, c, dl, g


def pack_psf(b, alpha, beta, a, c) -> np.ndarray:
    return np.concatenate([np.ravel(b), [alpha, beta], np.ravel(a), np.ravel(c)]).astype(np.float32)


def unpack_psf(p, S, N, f):
    F = f * N
    o = 0
    b = p[o:o + F * F].reshape(F, F); o += F * F
    alpha, beta = p[o], p[o + 1]; o += 2
    a = p[o:o + S]; o += S
    c = p[o:o + 2 * S].reshape(S, 2)
    return b, alpha, beta, a, c


# --- analytic profiles (input rendering only) ------------------------------------

def _grid(n, cx, cy, dtype=np.float64):
    y, x = np.mgrid[0:n, 0:n].astype(dtype)
    return x - cx, y - cy


def moffat_stamp(K, fwhm, beta, cx=None, cy=None, dtype=np.float64):
    """A Moffat-shaped image of size K, peak at (cx, cy) (default K//2), normalised to sum 1."""
    cx = K // 2 if cx is None else cx
    cy = K // 2 if cy is None else cy
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    x, y = _grid(K, cx, cy, dtype)
    img = (1.0 + (x * x + y * y) / alpha ** 2) ** (-beta)
    return (img / img.sum()).astype(dtype)


def moffat_stack(K, fwhm, beta, dtype=np.float32):
    """[E, K, K] Moffat PSFs (one per (fwhm, beta) pair), origin K//2, each normalised to 1."""
    fwhm = np.asarray(fwhm, dtype=np.float64).reshape(-1, 1, 1)
    beta = np.asarray(beta, dtype=np.float64).reshape(-1, 1, 1)
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    y, x = np.mgrid[0:K, 0:K].astype(np.float64)
    r2 = ((x - K // 2) ** 2 + (y - K // 2) ** 2)[None]
    img = (1.0 + r2 / alpha ** 2) ** (-beta)
    img /= img.sum(axis=(1, 2), keepdims=True)
    return img.astype(dtype)


def _sersic_bn(n):
    # Ciotti & Bertin (1999) asymptotic expansion of b_n
    return 2 * n - 1 / 3 + 4 / (405 * n) + 46 / (25515 * n ** 2) + 131 / (1148175 * n ** 3)


def sersic_image(n_pix, flux, n, re, cx=None, cy=None, q=1.0, ring_radius=None):
    """Sersic profile on an n_pix grid normalised so the grid sums to `flux`.
    With ring_radius, the profile is taken in |R - ring_radius| (a lensed arc / ring)."""
    cx = (n_pix - 1) / 2 if cx is None else cx
    cy = (n_pix - 1) / 2 if cy is None else cy
    x, y = _grid(n_pix, cx, cy)
    R = np.sqrt(x * x + (y / q) ** 2)
    if ring_radius is not None:
        R = np.abs(R - ring_radius)
    img = np.exp(-_sersic_bn(n) * ((R / re) ** (1.0 / n) - 1.0))
    return img * (flux / img.sum())


def gaussian_random_field(rng, n_pix, corr_len):
    """Unit-variance white noise smoothed by a Gaussian of std corr_len (FFT filtering of inputs)."""
    white = rng.standard_normal((n_pix, n_pix))
    k = np.fft.fftfreq(n_pix)
    kx, ky = np.meshgrid(k, k)
    filt = np.exp(-2 * (np.pi * corr_len) ** 2 * (kx * kx + ky * ky))
    field_ = np.real(np.fft.ifft2(np.fft.fft2(white) * filt))
    return field_ / (field_.std() + 1e-30)


def _data_stamp_sources(N, E, pos_data, amps, fwhm_data, beta):
    """Point sources rendered directly on the data grid as Moffat profiles.
    pos_data [E, M, 2] absolute data-pixel coordinates; amps [E, M]; fwhm/beta [E]."""
    y, x = np.mgrid[0:N, 0:N].astype(np.float32)
    out = np.zeros((E, N, N), dtype=np.float32)
    alpha = (fwhm_data / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))).astype(np.float32)
    for k in range(pos_data.shape[1]):
        dx = x[None] - pos_data[:, k, 0, None, None].astype(np.float32)
        dy = y[None] - pos_data[:, k, 1, None, None].astype(np.float32)
        a2 = (alpha ** 2)[:, None, None]
        b = beta.astype(np.float32)[:, None, None]
        prof = (1.0 + (dx * dx + dy * dy) / a2) ** (-b)
        norm = (b - 1.0) / (np.pi * a2)   # analytic unit flux of the profile
        out += amps[:, k, None, None].astype(np.float32) * prof * norm
    return out


def _noise(rng, model, sky):
    """Gaussian sky plus Poisson (gain 1) noise, sigma^2 = sky^2 + max(model, 0)."""
    sky = np.asarray(sky, dtype=np.float32)
    sky = sky.reshape(sky.shape + (1,) * (model.ndim - sky.ndim))
    var = sky * sky + np.maximum(model, 0.0)
    sigma = np.sqrt(var).astype(np.float32)
    d = (model + sigma * rng.standard_normal(model.shape, dtype=np.float32)).astype(np.float32)
    return d, sigma


def starlet_weights(J, sigma, f, E):
    """Synthetic per-scale prior weights: the starlet white-noise level per scale
    times the co-added noise level moved to the fine grid."""
    sig_eff = float(np.median(sigma)) / (f * np.sqrt(max(E, 1)))
    return (_STARLET_NOISE[:J - 1] * sig_eff).astype(np.float32)


# --- deconvolution workloads ----------------------------------------------------

def render_host(components, n_pix, scale=1.0, widen=0.0, rng=None, texture=0.0):
    """Sum of Sersic components on an n_pix grid.  Radii are given in fine
    pixels and multiplied by `scale` (1/f for the data grid); `widen` adds a
    width in quadrature (a crude stand-in for seeing on the data grid)."""
    img = np.zeros((n_pix, n_pix))
    for comp in components:
        re = np.sqrt((comp["re"] * scale) ** 2 + widen ** 2)
        ring = comp.get("ring")
        img += sersic_image(n_pix, comp["flux"], comp["n"], re, q=comp.get("q", 1.0),
                            ring_radius=None if ring is None else ring * scale)
    if texture and rng is not None:
        img *= 1.0 + texture * gaussian_random_field(rng, n_pix, 3.0)
    return img


def blurred_host_stack(components, N, f, fwhm_data, beta, sub=4):
    """The host seen through each epoch's seeing, on the data grid: the Sersic components
    integrated over each data pixel (sub x sub samples), convolved (FFT, 'same') with a unit-sum
    Moffat of the epoch's effective width (fwhm_data data pixels, exponent beta).  [E, N, N]."""
    from scipy.signal import fftconvolve
    fine = render_host(components, N * sub, scale=sub / f)
    sharp = fine.reshape(N, sub, N, sub).mean(axis=(1, 3)) * (sub * sub)
    out = np.empty((len(fwhm_data), N, N), dtype=np.float32)
    for i, (fw, b) in enumerate(zip(fwhm_data, beta)):
        kern = moffat_stamp(2 * N - 1, float(fw), float(b))
        out[i] = fftconvolve(sharp, kern, mode="same")
    return out


def make_deconv_field(rng, E, N, f, K, M, J, lam, *, psf_fwhm=(2.0, 3.0), psf_beta=(2.0, 4.0),
                      amp_range=(1e3, 1e4), pos_half=8.0, shift_std=0.1, host=None, sky=(5.0, 5.0),
                      light_curve=None, positions=None, texture=0.0, host_blur="mean"):
    F = f * N
    fwhm = rng.uniform(*psf_fwhm, size=E)
    beta = rng.uniform(*psf_beta, size=E)
    s = moffat_stack(K, fwhm, beta)
    if positions is None:
        positions = rng.uniform(-pos_half, pos_half, size=(M, 2))
    c = np.asarray(positions, dtype=np.float64).reshape(M, 2)
    delta = rng.normal(0.0, shift_std, size=(E, 2))
    if light_curve is None:
        base = np.exp(rng.uniform(np.log(amp_range[0]), np.log(amp_range[1]), size=M))
        a = base[None, :] * np.exp(rng.normal(0.0, 0.1, size=(E, M)))
    else:
        a = np.asarray(light_curve, dtype=np.float64).reshape(E, M)
    if host is None:
        host = [{"flux": 2e4, "n": 2.0, "re": 6.0}]
    # evaluation point: the host on the fine grid; data: the same components
    # drawn directly on the data grid, widened by the mean seeing (host_blur="mean") or seen
    # through each epoch's own seeing (host_blur="epoch", blurred_host_stack), plus point
    # sources drawn at data resolution with each epoch's effective width.
    h = render_host(host, F, rng=rng, texture=texture)
    fwhm_eff = np.sqrt(fwhm ** 2 + 4.0) / f
    centre = (N - 1) / 2.0
    pos = centre + c[None, :, :] + delta[:, None, :]
    if host_blur == "epoch":
        hd = blurred_host_stack(host, N, f, fwhm_eff, beta) if host else np.zeros((E, N, N), np.float32)
    else:
        hd = render_host(host, N, scale=1.0 / f, widen=float(np.mean(fwhm_eff)) / 2.355)[None].astype(np.float32)
    model = _data_stamp_sources(N, E, pos, a, fwhm_eff, beta) + hd
    sky_e = rng.uniform(*sky, size=E)
    d, sigma = _noise(rng, model, sky_e)
    W = starlet_weights(J, sigma, f, E)
    params = pack_deconv(h, a, c, delta, np.zeros(E))
    return DeconvField(E, N, f, K, M, J, float(lam), d, sigma, s.astype(np.float32), W, params,
                       meta={"fwhm": fwhm, "beta": beta, "sky": sky_e})


def config1(seed=None) -> DeconvField:
    """Plain joint deconvolution: 4 epochs of 32x32, f=2, K=64 Moffat PSFs
    (beta U[2,4], FWHM U[2,3] fine px), 2 point sources (amps log-U[1e3,1e4],
    positions within the central 16 px, shifts N(0, 0.1 px)), Sersic host (n=2,
    Re=6 fine px, flux 2e4), sky sigma 5 plus Poisson, 4 starlet scales, lambda 3."""
    rng = np.random.default_rng(BASE_SEED + 1 if seed is None else seed)
    return make_deconv_field(rng, E=4, N=32, f=2, K=64, M=2, J=4, lam=3.0)


def _drw(rng, n, tau, sf_inf, dt):
    """Damped random walk (AR(1) in magnitudes) sampled every dt days."""
    phi = np.exp(-dt / tau)
    sd = sf_inf / np.sqrt(2.0)
    m = np.empty(n)
    m[0] = rng.normal(0.0, sd)
    for t in range(1, n):
        m[t] = phi * m[t - 1] + sd * np.sqrt(1 - phi * phi) * rng.standard_normal()
    return m


def config3(seed=None, E=300, host_blur="mean") -> DeconvField:
    """Lensed-quasar light curves: 4 images at 1.2" (6 data px at 0.2"/px), 64x64
    stamps, f=2, 300 epochs each with a Moffat PSF (FWHM U[0.6,1.2]" = U[6,12]
    fine px, beta U[2,4]), ring Sersic arc plus lens galaxy, DRW fluxes, sky U[3,10]."""
    rng = np.random.default_rng(BASE_SEED + 3 if seed is None else seed)
    N, f, K, M = 64, 2, 64, 4
    F = f * N
    ang = np.array([0.0, 0.5, 1.0, 1.5]) * np.pi + rng.uniform(0, 2 * np.pi)
    rad = 6.0 + rng.uniform(-0.2, 0.2, size=4)
    pos = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    mag = np.stack([_drw(rng, E, 200.0, 0.2, 10.0) for _ in range(M)], axis=1)
    magn = np.array([1.0, 0.8, 0.6, 0.4])
    lc = 1e4 * magn[None, :] * 10 ** (-0.4 * mag)
    host = [{"flux": 2e4, "n": 1.0, "re": 1.5, "ring": 12.0}, {"flux": 3e4, "n": 3.0, "re": 8.0}]
    return make_deconv_field(rng, E=E, N=N, f=f, K=K, M=M, J=4, lam=2.0, psf_fwhm=(6.0, 12.0),
                             host=host, sky=(3.0, 10.0), light_curve=lc, positions=pos, host_blur=host_blur)


CONFIG4_SIZES = (32, 48, 64, 96, 128)


def config4_shapes(seed=None, n_fields=256):
    """Shapes of the uneven batch: (N, E, J) per field (N in {32..128}, E in [10,500], J in {4,5,6})."""
    rng = np.random.default_rng(BASE_SEED + 4 if seed is None else seed)
    Ns = rng.choice(CONFIG4_SIZES, size=n_fields)
    Es = rng.integers(10, 501, size=n_fields)
    Js = rng.integers(4, 7, size=n_fields)
    return [(int(n), int(e), int(j)) for n, e, j in zip(Ns, Es, Js)]


def config4_field(index, N, E, J, seed=None, host_blur="mean") -> DeconvField:
    """One SN + host field of the uneven batch: Gaussian-pulse SN light curve
    (peak 1e4 at a random epoch, width 20 epochs), two-Sersic host (n=4 bulge,
    n=1 disc) with a 10% random-field texture, f=2, K=64, 1 point source."""
    rng = np.random.default_rng((BASE_SEED + 4 if seed is None else seed) * 1000 + index + 1)
    f, K, M = 2, 64, 1
    F = f * N
    peak = rng.integers(0, E)
    t = np.arange(E)
    lc = 1e4 * np.exp(-0.5 * ((t - peak) / 20.0) ** 2) + 50.0
    re_scale = N / 64.0
    host = [{"flux": 3e4, "n": 4.0, "re": 4.0 * re_scale}, {"flux": 5e4, "n": 1.0, "re": 12.0 * re_scale, "q": 0.6}]
    pos = rng.uniform(-N / 8, N / 8, size=(1, 2))
    return make_deconv_field(rng, E=E, N=N, f=f, K=K, M=M, J=J, lam=2.0, psf_fwhm=(4.0, 10.0),
                             host=host, sky=(3.0, 10.0), light_curve=lc[:, None], positions=pos, texture=0.1,
                             host_blur=host_blur)


def point_source_field(seed, E, N, M, light_curve=None, positions=None, J=4) -> DeconvField:
    """Point sources on the sky background only (no extended source), f = 2, K = 64, Moffat PSFs
    of FWHM U[4, 10] fine px: the data then differ from the model only by how the point sources
    are sampled, so the extracted light curves measure the photometry itself.  light_curve [E][M]
    (default: log-uniform base fluxes with 10 % scatter), positions [M][2] in data pixels from the
    stamp centre (default: uniform within N/6)."""
    rng = np.random.default_rng(seed)
    return make_deconv_field(rng, E=E, N=N, f=2, K=64, M=M, J=J, lam=2.0, psf_fwhm=(4.0, 10.0), host=[],
                             sky=(3.0, 10.0), light_curve=light_curve, positions=positions, pos_half=N / 6)


def supernova_light_curve(E, peak_epoch, peak=1e4, width=20.0, floor=50.0):
    """Gaussian-pulse light curve [E][1] (the shape of the config-4 supernovae)."""
    t = np.arange(E)
    return (peak * np.exp(-0.5 * ((t - peak_epoch) / width) ** 2) + floor)[:, None]


def config4(seed=None, n_fields=256, fields=None) -> list[DeconvField]:
    shapes = config4_shapes(seed, n_fields)
    idx = range(len(shapes)) if fields is None else fields
    return [config4_field(i, *shapes[i], seed=seed) for i in idx]


def airy_psf_stack(rng, E, K, core_fwhm, aberr=0.05):
    """Airy-like core (2 J1(x)/x)^2 times (1 + aberr * random field), made asymmetric by the field; sum 1."""
    from scipy.special import j1
    y, x = np.mgrid[0:K, 0:K].astype(np.float64)
    r = np.sqrt((x - K // 2) ** 2 + (y - K // 2) ** 2)
    out = np.empty((E, K, K), dtype=np.float32)
    for i in range(E):
        scale = 1.028 * np.pi / (2 * 1.616) * 2.0 / core_fwhm[i]   # half max of the Airy core at FWHM/2
        z = r * scale
        core = np.where(z > 1e-8, (2.0 * j1(np.maximum(z, 1e-8)) / np.maximum(z, 1e-8)) ** 2, 1.0)
        img = core * (1.0 + aberr * gaussian_random_field(rng, K, 4.0)) + 1e-7 * np.exp(-r / (K / 6))
        img = np.maximum(img, 0.0)
        out[i] = (img / img.sum()).astype(np.float32)
    return out


def config5(seed=None, E=6, N=512) -> DeconvField:
    """JWST-like wide field: 6 frames of 512x512, f=3 (1536x1536 model grid),
    255x255 Airy-like PSFs with a random aberration, 40 compact clumps along an
    extended arc, 6 starlet scales."""
    rng = np.random.default_rng(BASE_SEED + 5 if seed is None else seed)
    f, K, M, J = 3, 255, 40, 6
    F = f * N
    s = airy_psf_stack(rng, E, K, rng.uniform(3.0, 5.0, size=E))
    comps = [{"flux": 5e6, "n": 1.0, "re": 6.0, "ring": F * 0.25, "q": 0.8}]
    # the arc plus a faint noise floor, as a reconstructed image carries everywhere (it also keeps
    # the starlet coefficients of the evaluation point away from exact zeros)
    host = render_host(comps, F) + 0.05 * rng.standard_normal((F, F))
    th = np.linspace(-0.6, 0.6, M) + rng.normal(0, 0.02, size=M)
    rad = N * 0.25 / 1.0
    pos = np.stack([rad * np.sin(th), rad * np.cos(th) * 0.8], axis=1)
    lc = np.exp(rng.uniform(np.log(2e3), np.log(2e4), size=M))[None, :] * np.ones((E, 1))
    fwhm = np.full(E, 4.0)
    beta = np.full(E, 3.0)
    delta = rng.normal(0.0, 0.05, size=(E, 2))
    hb = render_host(comps, N, scale=1.0 / f, widen=np.sqrt(4.0 ** 2 + 4.0) / f / 2.355)
    centre = (N - 1) / 2.0
    posd = centre + pos[None] + delta[:, None, :]
    model = _data_stamp_sources(N, E, posd, lc, np.sqrt(fwhm ** 2 + 4.0) / f, beta) + hb[None].astype(np.float32)
    sky = rng.uniform(3.0, 10.0, size=E)
    d, sigma = _noise(rng, model, sky)
    W = starlet_weights(J, sigma, f, E)
    params = pack_deconv(host, lc, pos, delta, np.zeros(E))
    return DeconvField(E, N, f, K, M, J, 2.0, d, sigma, s, W, params, meta={"sky": sky})


# --- PSF reconstruction workload -------------------------------------------------

def config2(seed=None, S=16, N=64) -> PsfProblem:
    """PSF reconstruction: 16 stars of 64x64, f=2 (128x128 narrow-PSF grid),
    Moffat beta 2.5, FWHM 3 fine px, plus a 5%-amplitude random-field pixel grid
    (correlation length 3 fine px); amplitudes log-U[1e4,1e5], centres U[-1,1]
    data px; 5 starlet scales, lambda 2."""
    rng = np.random.default_rng(BASE_SEED + 2 if seed is None else seed)
    f, J = 2, 5
    F = f * N
    beta = 2.5
    fwhm = 3.0
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    a = np.exp(rng.uniform(np.log(1e4), np.log(1e5), size=S))
    c = rng.uniform(-1.0, 1.0, size=(S, 2))
    envelope = moffat_stamp(F, fwhm, beta)      # unit-sum Moffat shape on the fine grid
    b = 0.05 * envelope * gaussian_random_field(rng, F, 3.0)
    # stars drawn at data resolution: Moffat of the effective width (narrow PSF
    # widened by the 2-px Gaussian) times a faint copy of the grid texture (the same
    # 5 % random field of correlation length 1.5 data px on every stamp)
    fwhm_eff = np.sqrt(fwhm ** 2 + 4.0) / f
    pos = (N - 1) / 2.0 + c
    texture = (1.0 + 0.05 * gaussian_random_field(rng, N, 1.5)).astype(np.float32)
    model = _data_stamp_sources(N, S, pos[:, None, :], a[:, None], np.full(S, fwhm_eff), np.full(S, beta))
    model = model * texture[None]
    d, sigma = _noise(rng, model, np.full(S, 10.0))
    W = starlet_weights(J, sigma, f, S)
    params = pack_psf(b, alpha, beta, a, c)
    return PsfProblem(S, N, f, J, 2.0, d, sigma, W, params, meta={"alpha": alpha, "beta": beta})


def small_deconv(seed, E=3, N=16, f=2, K=13, M=2, J=3, lam=1.0, **kw) -> DeconvField:
    """Small generic case (sizes the oracle finishes in well under a second)."""
    rng = np.random.default_rng(seed)
    kw.setdefault("pos_half", N / 6)
    return make_deconv_field(rng, E=E, N=N, f=f, K=K, M=M, J=J, lam=lam, **kw)


def small_psf(seed, S=3, N=16, f=2, J=3, lam=1.0) -> PsfProblem:
    rng = np.random.default_rng(seed)
    F = f * N
    beta = rng.uniform(2.0, 3.5)
    fwhm = rng.uniform(2.5, 4.0)
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    a = np.exp(rng.uniform(np.log(1e3), np.log(1e4), size=S))
    c = rng.uniform(-1.0, 1.0, size=(S, 2))
    b = 0.05 * moffat_stamp(F, fwhm, beta) * gaussian_random_field(rng, F, 2.0)
    pos = (N - 1) / 2.0 + c
    model = _data_stamp_sources(N, S, pos[:, None, :], a[:, None], np.full(S, np.sqrt(fwhm ** 2 + 4) / f),
                                np.full(S, beta))
    d, sigma = _noise(rng, model, np.full(S, 5.0))
    W = starlet_weights(J, sigma, f, S) * 1e-2
    return PsfProblem(S, N, f, J, float(lam), d, sigma, W, pack_psf(b, alpha, beta, a, c))
