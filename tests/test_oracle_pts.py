"""Pins for the oracle's point-source prior (Eq. 11, third term) and its lambda_pts estimate
(App. C): central differences, homogeneity and additivity, the mean over epochs, independence of
the per-epoch shifts, translation invariance, composition with an independent scipy starlet,
and closed forms of the estimate."""
import numpy as np
import pytest
import scipy.ndimage

import oracle
from paper_2402_08725_gb300 import synthetic as syn

B3 = np.array([1, 4, 6, 4, 1], dtype=np.float64) / 16.0


def _params(E, N, f, M, c, a, h=None, delta=None):
    F = f * N
    h = np.zeros((F, F)) if h is None else h
    a = np.broadcast_to(np.asarray(a, float), (E, M))
    delta = np.zeros((E, 2)) if delta is None else delta
    return syn.pack_deconv(h, a, np.asarray(c, float).reshape(M, 2), delta, np.zeros(E)).astype(np.float64)


def _details(x, J):
    out, c = [], x
    for j in range(J - 1):
        k = np.zeros(4 * (1 << j) + 1)
        k[:: 1 << j] = B3
        cn = scipy.ndimage.correlate1d(c, k, axis=1, mode="mirror")
        cn = scipy.ndimage.correlate1d(cn, k, axis=0, mode="mirror")
        out.append(c - cn)
        c = cn
    return np.array(out)


W4 = np.array([1.0, 0.6, 0.3])


def test_value_is_the_weighted_l1_of_the_mean_source_image():
    """Composition with a starlet written with scipy and the pinned Gaussian raster."""
    E, N, f, M, J, lam = 5, 24, 2, 2, 4, 0.7
    F = f * N
    rng = np.random.default_rng(1)
    a = rng.uniform(50, 150, (E, M))
    c = np.array([[-3.2, 1.1], [4.4, -2.7]])
    P = _params(E, N, f, M, c, a)
    a = P[F * F:F * F + E * M].reshape(E, M)  # the packed (float32-rounded) values
    c = P[F * F + E * M:F * F + E * M + 2 * M].reshape(M, 2)
    img = np.zeros((F, F))
    for k in range(M):
        u0 = 0.5 * (F - 1)
        img = oracle.add_gaussian(img, a[:, k].mean(), u0 + f * c[k, 0], u0 + f * c[k, 1])
    ref = lam * sum(W4[j] * np.abs(d).sum() for j, d in enumerate(_details(img, J)))
    v, _ = oracle.pts_prior(E, N, f, M, J, lam, W4, P, grad=False)
    assert abs(v - ref) <= 1e-12 * ref


def test_value_depends_on_the_mean_amplitude_only():
    E, N, f, M, J = 6, 20, 2, 1, 4
    c = [[0.3, -0.8]]
    base = oracle.pts_prior(E, N, f, M, J, 1.0, W4, _params(E, N, f, M, c, 100.0), grad=False)[0]
    ramp = np.linspace(40, 160, E)[:, None]  # same mean, different per-epoch values
    assert abs(oracle.pts_prior(E, N, f, M, J, 1.0, W4, _params(E, N, f, M, c, ramp), grad=False)[0] - base) \
        <= 1e-12 * base
    one = oracle.pts_prior(1, N, f, M, J, 1.0, W4, _params(1, N, f, M, c, 100.0), grad=False)[0]
    assert abs(one - base) <= 1e-12 * base  # a mean, not a sum, over epochs
    assert abs(oracle.pts_prior(E, N, f, M, J, 1.0, W4, _params(E, N, f, M, c, 250.0), grad=False)[0]
               - 2.5 * base) <= 1e-12 * base  # positively homogeneous in a
    assert oracle.pts_prior(E, N, f, M, J, 0.0, W4, _params(E, N, f, M, c, 100.0), grad=False)[0] == 0.0


def test_far_apart_sources_add_and_shifts_do_not_matter():
    E, N, f, J = 3, 40, 2, 3
    v1 = oracle.pts_prior(E, N, f, 1, J, 1.0, W4, _params(E, N, f, 1, [[-10.0, 0.0]], 80.0), grad=False)[0]
    v2 = oracle.pts_prior(E, N, f, 1, J, 1.0, W4, _params(E, N, f, 1, [[10.0, 0.0]], 30.0), grad=False)[0]
    v12 = oracle.pts_prior(E, N, f, 2, J, 1.0, W4, _params(E, N, f, 2, [[-10.0, 0.0], [10.0, 0.0]], [80.0, 30.0]),
                           grad=False)[0]
    assert abs(v12 - (v1 + v2)) <= 1e-10 * v12
    # a whole-pixel move of a source well inside the grid leaves the value unchanged
    v1s = oracle.pts_prior(E, N, f, 1, J, 1.0, W4, _params(E, N, f, 1, [[-9.0, 1.0]], 80.0), grad=False)[0]
    assert abs(v1s - v1) <= 1e-10 * v1
    # the per-epoch shifts move the epochs' point sources, not the mean image of the prior
    dl = np.random.default_rng(2).normal(0, 0.3, (E, 2))
    P = _params(E, N, f, 1, [[-10.0, 0.0]], 80.0, delta=dl)
    v, g = oracle.pts_prior(E, N, f, 1, J, 1.0, W4, P)
    assert abs(v - v1) <= 1e-12 * v1
    F = f * N
    od = F * F + E + 2
    assert np.all(g[od:od + 2 * E] == 0.0) and np.all(g[:F * F] == 0.0)


def test_gradient_central_differences():
    E, N, f, M, J = 4, 16, 2, 2, 3
    rng = np.random.default_rng(3)
    a = rng.uniform(20, 60, (E, M))
    P = _params(E, N, f, M, [[-1.37, 0.61], [2.21, -1.83]], a)
    F = f * N
    _, g = oracle.pts_prior(E, N, f, M, J, 0.9, W4, P)
    for k in list(range(F * F, F * F + E * M + 2 * M)):
        h = 1e-6 * max(1.0, abs(P[k]))
        pp, pm = P.copy(), P.copy()
        pp[k] += h
        pm[k] -= h
        fd = (oracle.pts_prior(E, N, f, M, J, 0.9, W4, pp, grad=False)[0]
              - oracle.pts_prior(E, N, f, M, J, 0.9, W4, pm, grad=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3), (k, fd, g[k])


# --- lambda_pts estimate (App. C) ------------------------------------------------------

def test_estimate_closed_forms():
    E, N, f, J, lam = 4, 32, 2, 4, 2.0
    F = f * N
    c = [[0.4, -0.3]]
    # one source, no extended flux: fbar = <a> r, the ratio is 1
    assert abs(oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, _params(E, N, f, 1, c, 90.0)) - lam) < 1e-12
    # two sources at the same place: the denominator sums what the numerator holds
    P = _params(E, N, f, 2, [[0.4, -0.3], [0.4, -0.3]], [30.0, 70.0])
    assert abs(oracle.lambda_pts_estimate(E, N, f, 2, J, lam, W4, P) - lam) < 1e-12
    # extended source far from the point source: norms add, the ratio is 1 again
    h = np.zeros((F, F))
    h[5:12, 6:14] = np.random.default_rng(4).uniform(1, 3, (7, 8))
    P = _params(E, N, f, 1, [[8.0, 8.0]], 90.0, h=h)
    assert abs(oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, P) - lam) < 1e-9
    # h cancels the point source exactly: fbar = 0, the ratio is -1
    P = _params(E, N, f, 1, c, 90.0)
    cx, cy = P[F * F + E], P[F * F + E + 1]
    P[:F * F] = -oracle.add_gaussian(np.zeros((F, F)), 90.0, 0.5 * (F - 1) + f * cx, 0.5 * (F - 1) + f * cy).ravel()
    assert abs(oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, P) + lam) < 1e-9
    # no point-source flux: 0
    assert oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, _params(E, N, f, 1, c, 0.0, h=h)) == 0.0


def test_estimate_below_lambda_when_channels_blend():
    """|A(h + a r)|_1 <= |A h|_1 + a |A r|_1 (triangle inequality): overlap lowers the ratio."""
    E, N, f, J, lam = 3, 24, 2, 4, 1.0
    F = f * N
    rng = np.random.default_rng(5)
    h = scipy.ndimage.gaussian_filter(rng.normal(0, 1, (F, F)), 2.0)
    P = _params(E, N, f, 1, [[0.0, 0.0]], 50.0, h=h)
    est = oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, P)
    assert -lam <= est < lam


def test_estimate_uses_the_epochs_shifted_sources():
    """Shifts of +-6 data px on alternate epochs split fbar into two separated half-flux copies:
    the norms still add up to the denominator's."""
    E, N, f, J, lam = 4, 48, 2, 3, 1.5
    dl = np.array([[6.0, 0.0], [-6.0, 0.0]] * 2)
    P = _params(E, N, f, 1, [[0.0, 0.0]], 60.0, delta=dl)
    assert abs(oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, P) - lam) < 1e-9
    # shifts small against the source: the copies overlap and the ratio drops below 1
    P = _params(E, N, f, 1, [[0.0, 0.0]], 60.0, delta=dl / 12.0)
    assert oracle.lambda_pts_estimate(E, N, f, 1, J, lam, W4, P) < lam - 1e-3
