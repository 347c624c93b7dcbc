"""The paper's accuracy metrics (sec. 3, the definitions before the time-series simulation):
astrometric precision, relative photometric accuracy and precision, and the mean absolute error
of a PSF.  Plain host arithmetic on arrays the caller provides (estimates read back from the
device and the generator's truth); nothing here runs on the GPU."""
from __future__ import annotations

import numpy as np


def astrometric_bias(c_true, c_est) -> np.ndarray:
    """b = (1/N) sum_k (c_k - c^_k) over the N positions (rows of 2-vectors)."""
    c_true = np.asarray(c_true, dtype=np.float64).reshape(-1, 2)
    c_est = np.asarray(c_est, dtype=np.float64).reshape(-1, 2)
    return np.mean(c_true - c_est, axis=0)


def p_astro(c_true, c_est) -> float:
    """P_astro = (1/N) sum_k || c_k - c^_k - b ||_2, the bias b removed (a sub-pixel bias can come
    from how the data were put on the pixel grid, so the metric measures the scatter)."""
    c_true = np.asarray(c_true, dtype=np.float64).reshape(-1, 2)
    c_est = np.asarray(c_est, dtype=np.float64).reshape(-1, 2)
    b = astrometric_bias(c_true, c_est)
    return float(np.mean(np.linalg.norm(c_true - c_est - b[None, :], axis=1)))


def _rel(f_true, f_est, mask):
    f_true = np.asarray(f_true, dtype=np.float64).ravel()
    f_est = np.asarray(f_est, dtype=np.float64).ravel()
    if mask is not None:
        keep = np.asarray(mask, dtype=bool).ravel()
        f_true, f_est = f_true[keep], f_est[keep]
    return (f_true - f_est) / f_est


def a_photo(f_true, f_est, mask=None) -> float:
    """A_photo = (1/N) sum_k (f_k - f^_k) / f^_k: the mean relative flux error (accuracy)."""
    return float(np.mean(_rel(f_true, f_est, mask)))


def p_photo(f_true, f_est, mask=None) -> float:
    """P_photo = (1/N) sum_k | (f_k - f^_k) / f^_k - A_photo |: the mean absolute scatter of the
    relative flux errors about their mean (precision)."""
    r = _rel(f_true, f_est, mask)
    return float(np.mean(np.abs(r - np.mean(r))))


def mae_psf(psf_true, psf_est) -> float:
    """MAE_PSF = || PSF - PSF^ ||_1 over the pixels of the two (equally sampled) PSF images."""
    return float(np.sum(np.abs(np.asarray(psf_true, dtype=np.float64) - np.asarray(psf_est, dtype=np.float64))))
