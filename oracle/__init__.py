"""FP64 CPU oracle for the STARRED loss and gradient (arXiv 2402.08725).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library in ``paper_2402_08725_gb300`` and its binding) never imports
it, and the two share no code: the arithmetic lives in ``starred_oracle.c``
(plain C, double precision, literal operator order) and this module only
marshals numpy arrays into it.

Every function converts its inputs to float64 first, so the oracle evaluates
the exact loss of the float32 values the GPU receives.

Functions and the passages they follow:
  conv_same / conv_same_adjoint   S_i, the narrow-PSF convolution (Eq. 8, Eq. 10)
  downsample / downsample_adjoint D, the block-sum subsampling (Eq. 1)
  starlet_analysis / _adjoint     Phi^T, the starlet transform of the prior (Eq. 6)
  starlet_prior                   lambda ||W o Phi^T h||_1 and its subgradient (Eq. 6, Eq. 11)
  deconv_model / deconv_loss_grad the two-channel multi-epoch model and loss (Eq. 9-11)
  translate / _adjoint            the extended channel moved with an epoch's shift (sec. 5; bilinear)
  warp / _adjoint                 an epoch's frame rotated about the grid centre and shifted (sec. 5)
  moffat                          the analytic part of the narrow PSF (Eq. 2)
  psf_model / psf_loss_grad       PSF reconstruction (Eq. 2-4, Eq. 7)
  optim_step                      AdaBelief / Adam update used by the optimiser (sec. 2.4)
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "starred_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def _lib_path() -> str:
    with open(_SRC, "rb") as fh:
        digest = hashlib.sha1(fh.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"liborc_{os.uname().machine}_{digest}.so")


def build() -> str:
    """Compile the C oracle (gcc, -O2, OpenMP) if it is not built yet; return the .so path."""
    path = _lib_path()
    if os.path.exists(path):
        return path
    os.makedirs(_BUILD, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sig = {
            "orc_version": ([], i),
            "orc_max_threads": ([], i),
            "orc_set_threads": ([i], None),
            "orc_conv_same": ([i, i, _dp, _dp, _dp], i),
            "orc_conv_same_adjoint": ([i, i, _dp, _dp, _dp], i),
            "orc_downsample": ([i, i, _dp, _dp], i),
            "orc_downsample_adjoint": ([i, i, _dp, _dp], i),
            "orc_starlet_valid": ([i, i], i),
            "orc_starlet_analysis": ([i, i, _dp, _dp], i),
            "orc_starlet_adjoint": ([i, i, _dp, _dp], i),
            "orc_starlet_prior": ([i, i, d, _dp, _dp, _dp, _dp], i),
            "orc_starlet_prior_map": ([i, i, d, _dp, _dp, _dp, _dp], i),
            "orc_psf_loss_grad_map": ([i, i, i, i, d, _dp, _dp, _dp, _dp, _dp, _dp, i], i),
            "orc_pts_prior_map": ([i, i, i, i, i, d, _dp, _dp, _dp, _dp], i),
            "orc_add_gaussian": ([i, d, d, d, _dp], i),
            "orc_deconv_param_count": ([i, i, i, i], sz),
            "orc_deconv_model": ([i, i, i, i, i, _dp, _dp, _dp], i),
            "orc_deconv_loss_grad": ([i, i, i, i, i, i, d, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, i], i),
            "orc_deconv_loss_grad_shifted": ([i, i, i, i, i, i, d, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, i], i),
            "orc_translate": ([i, d, d, _dp, _dp], i),
            "orc_warp": ([i, d, d, d, _dp, _dp], i),
            "orc_warp_adjoint": ([i, d, d, d, _dp, _dp], i),
            "orc_deconv_model_ex": ([i, i, i, i, i, _dp, _dp, _dp, i, _dp], i),
            "orc_deconv_loss_grad_ex": ([i, i, i, i, i, i, d, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, i, i, _dp, _dp],
                                        i),
            "orc_translate_adjoint": ([i, d, d, _dp, _dp], i),
            "orc_moffat": ([i, d, d, _dp, _dp, _dp], i),
            "orc_psf_param_count": ([i, i, i], sz),
            "orc_psf_model": ([i, i, i, _dp, _dp], i),
            "orc_psf_loss_grad": ([i, i, i, i, d, _dp, _dp, _dp, _dp, _dp, _dp, i], i),
            "orc_optim_step": ([i, ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.c_long, _dp, d, d, d, _dp, _dp], i),
            "orc_pts_prior": ([i, i, i, i, i, d, _dp, _dp, _dp, _dp], i),
            "orc_lambda_pts_estimate": ([i, i, i, i, i, d, _dp, _dp, _dp], i),
            "orc_philox4x64": ([ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64)], None),
            "orc_normal": ([ctypes.c_uint64, ctypes.c_uint64], d),
            "orc_noise_weights": ([i, i, i, i, i, _dp, _dp, i, ctypes.c_uint64, _dp, _dp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of later oracle calls (timing only; results do not depend on it)."""
    _load().orc_set_threads(int(n))


# --- building blocks -------------------------------------------------------

def conv_same(x, s):
    """S: out[u] = sum_q s[q] x[u - q + o], o = K//2, zero padding, F x F output."""
    x, s = _f64(x), _f64(s)
    F, K = x.shape[0], s.shape[0]
    out = np.empty((F, F))
    _check(_load().orc_conv_same(F, K, _ptr(x), _ptr(s), _ptr(out)), "conv_same")
    return out


def conv_same_adjoint(y, s):
    y, s = _f64(y), _f64(s)
    F, K = y.shape[0], s.shape[0]
    out = np.empty((F, F))
    _check(_load().orc_conv_same_adjoint(F, K, _ptr(y), _ptr(s), _ptr(out)), "conv_same_adjoint")
    return out


def translate(h, sx, sy):
    """The fine image moved by (sx, sy) fine pixels: out(u) = h(u - s), bilinear, zero outside
    (the extended channel moved with an epoch's shift, sec. 5; the interpolation is a reading)."""
    h = _f64(h)
    F = h.shape[0]
    out = np.empty((F, F))
    _check(_load().orc_translate(F, float(sx), float(sy), _ptr(h), _ptr(out)), "translate")
    return out


def warp(h, theta, sx=0.0, sy=0.0):
    """h seen in a frame rotated by theta (radians) about the grid centre and shifted by (sx, sy)
    fine pixels: out(u) = h at u0 + R^T (u - u0 - s), bilinear, zero outside (orc_warp)."""
    h = _f64(h)
    F = h.shape[0]
    out = np.empty_like(h)
    _check(_load().orc_warp(F, float(theta), float(sx), float(sy), _ptr(h), _ptr(out)), "warp")
    return out


def warp_adjoint(g, theta, sx=0.0, sy=0.0):
    """Transpose of warp."""
    g = _f64(g)
    F = g.shape[0]
    out = np.empty_like(g)
    _check(_load().orc_warp_adjoint(F, float(theta), float(sx), float(sy), _ptr(g), _ptr(out)), "warp_adjoint")
    return out


def translate_adjoint(g, sx, sy):
    g = _f64(g)
    F = g.shape[0]
    out = np.empty((F, F))
    _check(_load().orc_translate_adjoint(F, float(sx), float(sy), _ptr(g), _ptr(out)), "translate_adjoint")
    return out


def downsample(x, f: int):
    x = _f64(x)
    N = x.shape[0] // f
    out = np.empty((N, N))
    _check(_load().orc_downsample(N, f, _ptr(x), _ptr(out)), "downsample")
    return out


def downsample_adjoint(e, f: int):
    e = _f64(e)
    N = e.shape[0]
    out = np.empty((N * f, N * f))
    _check(_load().orc_downsample_adjoint(N, f, _ptr(e), _ptr(out)), "downsample_adjoint")
    return out


def starlet_valid(F: int, J: int) -> bool:
    return bool(_load().orc_starlet_valid(F, J))


def starlet_analysis(h, J: int):
    """Planes [w_1, ..., w_{J-1}, c_{J-1}] of the B3 a trous transform of h."""
    h = _f64(h)
    F = h.shape[0]
    out = np.empty((J, F, F))
    _check(_load().orc_starlet_analysis(F, J, _ptr(h), _ptr(out)), "starlet_analysis")
    return out


def starlet_adjoint(y):
    y = _f64(y)
    J, F = y.shape[0], y.shape[1]
    out = np.empty((F, F))
    _check(_load().orc_starlet_adjoint(F, J, _ptr(y), _ptr(out)), "starlet_adjoint")
    return out


def starlet_prior(h, J: int, lam: float, W, grad: bool = True):
    """lam sum_j W_j ||w_j||_1; W of shape (J-1,) per scale, or (J-1, F, F) per coefficient."""
    h, W = _f64(h), _f64(W)
    F = h.shape[0]
    p = np.zeros(1)
    g = np.empty((F, F)) if grad else None
    if W.ndim == 3:
        if W.shape != (J - 1, F, F):
            raise ValueError(f"weight map of shape {W.shape}, expected {(J - 1, F, F)}")
        _check(_load().orc_starlet_prior_map(F, J, float(lam), _ptr(W), _ptr(h), _ptr(p), _ptr(g)), "starlet_prior")
    else:
        _check(_load().orc_starlet_prior(F, J, float(lam), _ptr(W), _ptr(h), _ptr(p), _ptr(g)), "starlet_prior")
    return (float(p[0]), g) if grad else float(p[0])


def add_gaussian(img, amp: float, ux: float, uy: float):
    img = _f64(img).copy()
    _check(_load().orc_add_gaussian(img.shape[0], float(amp), float(ux), float(uy), _ptr(img)), "add_gaussian")
    return img


# --- deconvolution (Eq. 9-11) ----------------------------------------------

def deconv_param_count(E: int, N: int, f: int, M: int) -> int:
    return int(_load().orc_deconv_param_count(E, N, f, M))


def deconv_model(E, N, f, K, M, s, params, shifted=False, theta=None):
    """Model of every epoch; shifted / theta as in deconv_loss_grad."""
    s, params = _f64(s), _f64(params)
    out = np.empty((E, N, N))
    if not shifted and theta is None:
        _check(_load().orc_deconv_model(E, N, f, K, M, _ptr(s), _ptr(params), _ptr(out)), "deconv_model")
        return out
    th = None if theta is None else _f64(theta)
    if th is not None and th.size != E:
        raise ValueError(f"theta has {th.size} values, expected {E}")
    _check(_load().orc_deconv_model_ex(E, N, f, K, M, _ptr(s), _ptr(params), _ptr(out), int(bool(shifted)),
                                       _ptr(th) if th is not None else None), "deconv_model")
    return out


def deconv_loss_grad(E, N, f, K, M, J, lam, d, sigma, s, W, params, grad=True, nthreads=0, shifted=False,
                     theta=None):
    """Return (loss, parts[chi2, prior], grad or None, chi2 per epoch).  shifted=True moves the
    extended channel h by each epoch's shift f * delta_i (translate) before the convolution;
    theta (E angles in radians) rotates each epoch's frame about the grid centre (warp).  W of
    shape (J-1,) weights each scale, of shape (J-1, F, F) each coefficient."""
    d, sigma, s, W, params = _f64(d), _f64(sigma), _f64(s), _f64(W), _f64(params)
    n = deconv_param_count(E, N, f, M)
    if params.size != n:
        raise ValueError(f"params has {params.size} values, expected {n}")
    parts = np.zeros(2)
    g = np.empty(n) if grad else None
    chi = np.empty(E)
    if theta is not None or W.ndim == 3:
        th = None if theta is None else _f64(theta)
        if th is not None and th.size != E:
            raise ValueError(f"theta has {th.size} values, expected {E}")
        wmap = W if W.ndim == 3 else None
        if wmap is not None and wmap.shape != (J - 1, f * N, f * N):
            raise ValueError(f"weight map of shape {wmap.shape}, expected {(J - 1, f * N, f * N)}")
        rc = _load().orc_deconv_loss_grad_ex(E, N, f, K, M, J, float(lam), _ptr(d), _ptr(sigma), _ptr(s),
                                             _ptr(W if wmap is None else np.zeros(J - 1)), _ptr(params), _ptr(parts),
                                             _ptr(g), _ptr(chi), int(nthreads), int(bool(shifted)), _ptr(th),
                                             _ptr(wmap))
    else:
        fn = _load().orc_deconv_loss_grad_shifted if shifted else _load().orc_deconv_loss_grad
        rc = fn(E, N, f, K, M, J, float(lam), _ptr(d), _ptr(sigma), _ptr(s), _ptr(W), _ptr(params), _ptr(parts),
                _ptr(g), _ptr(chi), int(nthreads))
    _check(rc, "deconv_loss_grad")
    return float(parts.sum()), parts, g, chi


# --- PSF reconstruction (Eq. 2-4, 7) ----------------------------------------

def pts_prior(E, N, f, M, J, lam_pts, W, params, grad=True):
    """Point-source prior of Eq. 11 (third term): (value, gradient over the packed deconvolution
    parameters, zero outside the a and c blocks)."""
    P = _f64(params)
    Wv = _f64(W)
    v = ctypes.c_double()
    g = np.zeros_like(P) if grad else None
    fn = _load().orc_pts_prior_map if Wv.ndim == 3 else _load().orc_pts_prior
    _check(fn(int(E), int(N), int(f), int(M), int(J), float(lam_pts), _ptr(Wv), _ptr(P),
              ctypes.byref(v), _ptr(g) if grad else None), "pts_prior")
    return v.value, g


def lambda_pts_estimate(E, N, f, M, J, lam, W, params) -> float:
    """lambda_pts from a model by the ratio of App. C."""
    out = ctypes.c_double()
    _check(_load().orc_lambda_pts_estimate(int(E), int(N), int(f), int(M), int(J), float(lam), _ptr(_f64(W)),
                                           _ptr(_f64(params)), ctypes.byref(out)), "lambda_pts_estimate")
    return out.value


def moffat(F: int, alpha: float, beta: float):
    m, da, db = np.empty((F, F)), np.empty((F, F)), np.empty((F, F))
    _check(_load().orc_moffat(F, float(alpha), float(beta), _ptr(m), _ptr(da), _ptr(db)), "moffat")
    return m, da, db


def psf_param_count(S: int, N: int, f: int) -> int:
    return int(_load().orc_psf_param_count(S, N, f))


def psf_model(S, N, f, params):
    params = _f64(params)
    out = np.empty((S, N, N))
    _check(_load().orc_psf_model(S, N, f, _ptr(params), _ptr(out)), "psf_model")
    return out


def psf_loss_grad(S, N, f, J, lam, t, sigma, W, params, grad=True, nthreads=0):
    t, sigma, W, params = _f64(t), _f64(sigma), _f64(W), _f64(params)
    n = psf_param_count(S, N, f)
    if params.size != n:
        raise ValueError(f"params has {params.size} values, expected {n}")
    parts = np.zeros(2)
    g = np.empty(n) if grad else None
    fn = _load().orc_psf_loss_grad_map if W.ndim == 3 else _load().orc_psf_loss_grad
    rc = fn(S, N, f, J, float(lam), _ptr(t), _ptr(sigma), _ptr(W), _ptr(params), _ptr(parts), _ptr(g), int(nthreads))
    _check(rc, "psf_loss_grad")
    return float(parts.sum()), parts, g


# --- optimiser ----------------------------------------------------------------

ADABELIEF, ADAM = 0, 1


def optim_step(kind, theta, g, m, v, t, lr, beta1, beta2, eps, lo, hi):
    """One in-place update of theta, m, v (all float64 arrays). t is 1-based."""
    for a in (theta, g, m, v, lr, lo, hi):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("optim_step wants contiguous float64 arrays")
    rc = _load().orc_optim_step(int(kind), theta.size, _ptr(theta), _ptr(g), _ptr(m), _ptr(v), int(t), _ptr(lr),
                                float(beta1), float(beta2), float(eps), _ptr(lo), _ptr(hi))
    _check(rc, "optim_step")


# --- noise propagation (sec. 2.3, App. B) ------------------------------------

def philox4x64(counter, key):
    """One Philox4x64-10 block (Salmon et al. 2011): four 64-bit words."""
    c = (ctypes.c_uint64 * 4)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in counter])
    k = (ctypes.c_uint64 * 2)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in key])
    out = (ctypes.c_uint64 * 4)()
    _load().orc_philox4x64(c, k, out)
    return [int(v) for v in out]


def normal(seed: int, n: int) -> float:
    """Standard normal number n of stream `seed` (Philox4x64-10 + Box-Muller on 24-bit uniforms)."""
    return float(_load().orc_normal(int(seed), int(n)))


def noise_weights(N, f, K, J, sigma, s1, n_real, seed):
    """Monte Carlo starlet weights of sec. 2.3 from n_real realisations of S_1^T (C^)^-1 dd:
    (W_scale [J-1], the pooled standard deviation of each detail scale, and W_map [J-1][fN][fN],
    the standard deviation of each coefficient)."""
    sigma = _f64(sigma).reshape(-1, N, N)
    s1 = _f64(s1).reshape(K, K)
    F = f * N
    W = np.empty((J - 1, F, F))
    Ws = np.empty(J - 1)
    _check(_load().orc_noise_weights(int(N), int(f), int(K), int(J), int(sigma.shape[0]), _ptr(sigma), _ptr(s1),
                                     int(n_real), ctypes.c_uint64(int(seed)), _ptr(W), _ptr(Ws)), "noise_weights")
    return Ws, W
