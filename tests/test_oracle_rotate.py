"""Pins of the oracle's rotated frames (sec. 5 names rotations between frames; no equation fixes
them, so the reading is: epoch i's frame is the reference frame rotated by theta_i about the grid
centre and, when the extended channel moves with the shifts, shifted by f delta_i; bilinear
interpolation, zero outside; point sources at u0 + f (R c_k + delta_i)).  scipy's linear affine
transform, the quarter turn as np.rot90, zero angle as the translation, the dot-product adjoint,
the two channels turning the same way, and central differences of the loss."""
import numpy as np
import pytest

import oracle
from paper_2402_08725_gb300 import synthetic as syn

ndimage = pytest.importorskip("scipy.ndimage")


def _affine_ref(h, theta, sx, sy):
    """scipy's order-1 affine transform with zero fill: output index (oy, ox) reads the input at
    A (oy, ox) + b, A and b the inverse of the frame map (rotation about u0, then the shift)."""
    F = h.shape[0]
    u0 = 0.5 * (F - 1)
    ct, st = np.cos(theta), np.sin(theta)
    A = np.array([[ct, -st], [st, ct]])
    b = np.array([u0, u0]) - A @ np.array([u0 + sy, u0 + sx])
    return ndimage.affine_transform(h, A, offset=b, order=1, mode="grid-constant", cval=0.0, prefilter=False)


@pytest.mark.parametrize("theta,sx,sy", [(0.37, 0.8, -1.3), (-1.1, 0.0, 0.0), (2.9, -2.4, 0.6), (0.05, 4.2, 3.3)])
def test_warp_is_the_linear_affine_transform_with_zero_fill(theta, sx, sy):
    rng = np.random.default_rng(11)
    h = rng.normal(size=(24, 24))
    np.testing.assert_allclose(oracle.warp(h, theta, sx, sy), _affine_ref(h, theta, sx, sy), rtol=0, atol=1e-12)


def test_quarter_turn_is_rot90_and_zero_angle_is_the_translation():
    rng = np.random.default_rng(12)
    h = rng.normal(size=(16, 16))
    # out(x0 + dx, y0 + dy) = h(x0 + dy, y0 - dx): in [row][column] order np.rot90 clockwise
    np.testing.assert_allclose(oracle.warp(h, np.pi / 2), np.rot90(h, -1), rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.warp(h, np.pi), h[::-1, ::-1], rtol=0, atol=1e-12)
    for sx, sy in [(0.3, -0.7), (-1.6, 2.25)]:
        np.testing.assert_allclose(oracle.warp(h, 0.0, sx, sy), oracle.translate(h, sx, sy), rtol=0, atol=1e-12)


def test_warp_adjoint_dot_product():
    rng = np.random.default_rng(13)
    for theta, sx, sy in [(0.4, -1.3, 0.2), (-2.7, 0.6, 1.9), (1.0, 0.0, 0.0)]:
        h, g = rng.normal(size=(21, 21)), rng.normal(size=(21, 21))
        lhs = float(np.sum(oracle.warp(h, theta, sx, sy) * g))
        rhs = float(np.sum(h * oracle.warp_adjoint(g, theta, sx, sy)))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_both_channels_turn_the_same_way():
    """A quarter turn of every frame equals the unrotated model of the turned scene: h as
    np.rot90(h, -1) and each source at R c = (-c_y, c_x)."""
    fd = syn.small_deconv(seed=43, E=2, N=12, f=2, K=7, M=2, J=3, lam=0.7)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    P = syn.pack_deconv(h, a, c, dl, gm).astype(np.float64)
    turned = syn.pack_deconv(np.rot90(h, -1), a, np.stack([-c[:, 1], c[:, 0]], axis=1), dl, gm).astype(np.float64)
    m1 = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, P, theta=np.full(fd.E, np.pi / 2))
    m0 = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, turned)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-9 * np.abs(m0).max())


def _field():
    fd = syn.small_deconv(seed=44, E=3, N=12, f=2, K=7, M=2, J=3, lam=0.7)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    dl = np.array([[0.13, -0.21], [-0.32, 0.17], [0.41, 0.09]])
    return fd, syn.pack_deconv(h, a, c, dl, gm).astype(np.float64), np.array([0.21, -0.47, 1.3])


@pytest.mark.parametrize("shifted", [False, True])
def test_rotated_loss_central_differences(shifted):
    """Shifts, source positions and amplitudes, a sample of h pixels and the backgrounds."""
    fd, P, theta = _field()
    args = (fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W)
    L, _, g, _ = oracle.deconv_loss_grad(*args, P, shifted=shifted, theta=theta)
    F = fd.F
    oa = F * F
    oc = oa + fd.E * fd.M
    od = oc + 2 * fd.M
    og = od + 2 * fd.E
    idx = list(range(od, od + 2 * fd.E)) + list(range(oc, oc + 2 * fd.M)) + [oa, oa + 3] + \
        [5 * F + 7, 11 * F + 12, 13 * F + 3] + [og, og + 2]
    for j in idx:
        hstep = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += hstep
        Pm[j] -= hstep
        Lp = oracle.deconv_loss_grad(*args, Pp, grad=False, shifted=shifted, theta=theta)[0]
        Lm = oracle.deconv_loss_grad(*args, Pm, grad=False, shifted=shifted, theta=theta)[0]
        fdv = (Lp - Lm) / (2 * hstep)
        assert abs(fdv - g[j]) <= 1e-6 * max(abs(g[j]), 1.0) + 1e-6, (j, fdv, g[j])
