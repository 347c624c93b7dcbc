"""Pins of the oracle's per-coefficient prior weights W_j(u) (sec. 2.3 and App. B propagate the
noise to a map per scale): one coefficient weighted alone gives lam |w_j(u)| of the pinned starlet
(asymmetric position, every plane), the prior is linear in the map, a map constant per plane is
the per-scale prior, and central differences of the prior and of the deconvolution and PSF losses."""
import numpy as np
import pytest

import oracle
from paper_2402_08725_gb300 import synthetic as syn


def test_one_weighted_coefficient_is_its_magnitude():
    rng = np.random.default_rng(21)
    F, J, lam = 32, 4, 1.7
    h = rng.normal(size=(F, F))
    planes = oracle.starlet_analysis(h, J)
    for j, (y, x) in [(0, (3, 17)), (1, (20, 5)), (2, (11, 29))]:
        Wm = np.zeros((J - 1, F, F))
        Wm[j, y, x] = 1.0
        v = oracle.starlet_prior(h, J, lam, Wm, grad=False)
        assert abs(v - lam * abs(planes[j][y, x])) <= 1e-12 * max(1.0, abs(v))


def test_map_is_linear_and_constant_planes_are_the_per_scale_prior():
    rng = np.random.default_rng(22)
    F, J, lam = 24, 4, 0.9
    h = rng.normal(size=(F, F))
    W = np.array([0.3, 0.7, 1.9])
    v0, g0 = oracle.starlet_prior(h, J, lam, W)
    v1, g1 = oracle.starlet_prior(h, J, lam, np.broadcast_to(W[:, None, None], (J - 1, F, F)).copy())
    assert abs(v1 - v0) <= 1e-12 * abs(v0)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-12 * np.abs(g0).max())
    A, B = rng.uniform(0, 1, (J - 1, F, F)), rng.uniform(0, 1, (J - 1, F, F))
    va, ga = oracle.starlet_prior(h, J, lam, A)
    vb, gb = oracle.starlet_prior(h, J, lam, B)
    vab, gab = oracle.starlet_prior(h, J, lam, A + B)
    assert abs(vab - va - vb) <= 1e-12 * abs(vab)
    np.testing.assert_allclose(gab, ga + gb, rtol=0, atol=1e-12 * np.abs(gab).max())


def test_map_prior_and_losses_central_differences():
    rng = np.random.default_rng(23)
    fd = syn.small_deconv(seed=24, E=2, N=12, f=2, K=7, M=1, J=3, lam=1.2)
    F = fd.F
    Wm = rng.uniform(0.2, 2.0, (fd.J - 1, F, F)) * np.asarray(fd.W, dtype=np.float64)[:, None, None]
    P = fd.params.astype(np.float64)
    args = (fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, Wm)
    L, _, g, _ = oracle.deconv_loss_grad(*args, P)
    L0, _, _, _ = oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W, P)
    assert L != L0
    for j in [3 * F + 5, 10 * F + 17, 20 * F + 2, F * F + 1]:
        hs = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += hs
        Pm[j] -= hs
        fdv = (oracle.deconv_loss_grad(*args, Pp, grad=False)[0] - oracle.deconv_loss_grad(*args, Pm, grad=False)[0]) / (2 * hs)
        # central-difference rounding: about 1e-16 L / hs
        assert abs(fdv - g[j]) <= 1e-6 * max(abs(g[j]), 1.0) + 4e-16 * abs(L) / hs, (j, fdv, g[j])
    pb = syn.small_psf(25, S=2, N=12, f=2, J=3, lam=1.0)
    Fp = pb.f * pb.N
    Wp = rng.uniform(0.2, 2.0, (pb.J - 1, Fp, Fp)) * np.asarray(pb.W, dtype=np.float64)[:, None, None]
    Q = pb.params.astype(np.float64)
    pa = (pb.S, pb.N, pb.f, pb.J, pb.lam, pb.t, pb.sigma, Wp)
    Lq, _, gq = oracle.psf_loss_grad(*pa, Q)
    for j in [2 * Fp + 3, 9 * Fp + 14]:
        hs = 1e-7
        Qp, Qm = Q.copy(), Q.copy()
        Qp[j] += hs
        Qm[j] -= hs
        fdv = (oracle.psf_loss_grad(*pa, Qp, grad=False)[0] - oracle.psf_loss_grad(*pa, Qm, grad=False)[0]) / (2 * hs)
        assert abs(fdv - gq[j]) <= 1e-5 * max(abs(gq[j]), 1.0), (j, fdv, gq[j])


def test_point_source_prior_with_a_map_central_differences():
    rng = np.random.default_rng(26)
    fd = syn.small_deconv(seed=27, E=3, N=12, f=2, K=7, M=2, J=3, lam=1.0)
    F = fd.F
    Wm = rng.uniform(0.2, 2.0, (fd.J - 1, F, F))
    P = fd.params.astype(np.float64)
    v, g = oracle.pts_prior(fd.E, fd.N, fd.f, fd.M, fd.J, 0.8, Wm, P)
    oa = F * F
    for j in [oa, oa + 3, oa + fd.E * fd.M, oa + fd.E * fd.M + 3]:
        hs = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += hs
        Pm[j] -= hs
        fdv = (oracle.pts_prior(fd.E, fd.N, fd.f, fd.M, fd.J, 0.8, Wm, Pp, grad=False)[0]
               - oracle.pts_prior(fd.E, fd.N, fd.f, fd.M, fd.J, 0.8, Wm, Pm, grad=False)[0]) / (2 * hs)
        assert abs(fdv - g[j]) <= 1e-6 * max(abs(g[j]), 1.0) + 1e-6, (j, fdv, g[j])
