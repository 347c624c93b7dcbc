"""Pins of the oracle's moved extended channel (h translated by each epoch's shift f * delta_i, the
frame shifts of sec. 5, with bilinear interpolation as the reading of the interpolation the paper
leaves open): scipy's linear shift with zero fill, whole-pixel shifts as rolls, the dot-product
adjoint, and central differences of the loss with the moved channel."""
import numpy as np
import pytest

import oracle
from paper_2402_08725_gb300 import synthetic as syn

ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("sx,sy", [(0.3, -0.7), (-1.6, 2.25), (3.0, -2.0), (0.0, 0.0), (-0.95, 0.05)])
def test_translate_is_the_linear_shift_with_zero_fill(sx, sy):
    rng = np.random.default_rng(5)
    h = rng.normal(size=(23, 23))
    ref = ndimage.shift(h, (sy, sx), order=1, mode="grid-constant", cval=0.0, prefilter=False)
    np.testing.assert_allclose(oracle.translate(h, sx, sy), ref, rtol=0, atol=1e-12)


def test_whole_pixel_shift_is_a_roll_with_zero_fill():
    rng = np.random.default_rng(6)
    h = rng.normal(size=(16, 16))
    out = oracle.translate(h, 3.0, -2.0)   # out(u) = h(u - s): content moves right 3, up 2
    ref = np.zeros_like(h)
    ref[:-2, 3:] = h[2:, :-3]
    np.testing.assert_array_equal(out, ref)
    np.testing.assert_array_equal(oracle.translate(h, 0.0, 0.0), h)


def test_translate_adjoint_dot_product():
    rng = np.random.default_rng(7)
    for sx, sy in [(0.4, -1.3), (-2.7, 0.6), (5.5, 5.5)]:
        h, g = rng.normal(size=(19, 19)), rng.normal(size=(19, 19))
        lhs = float(np.sum(oracle.translate(h, sx, sy) * g))
        rhs = float(np.sum(h * oracle.translate_adjoint(g, sx, sy)))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def _field():
    fd = syn.small_deconv(seed=41, E=3, N=12, f=2, K=7, M=2, J=3, lam=0.7)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    dl = np.array([[0.13, -0.21], [-0.32, 0.17], [0.41, 0.09]])   # f delta away from whole pixels
    return fd, syn.pack_deconv(h, a, c, dl, gm).astype(np.float64)


def test_zero_shift_moves_nothing():
    fd, P = _field()
    h, a, c, dl, gm = syn.unpack_deconv(P.copy(), fd.E, fd.N, fd.f, fd.M)
    P0 = syn.pack_deconv(h, a, c, np.zeros_like(dl), gm).astype(np.float64)
    args = (fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W, P0)
    L0, _, g0, _ = oracle.deconv_loss_grad(*args)
    L1, _, g1, _ = oracle.deconv_loss_grad(*args, shifted=True)
    assert abs(L0 - L1) <= 1e-12 * abs(L0)
    F = fd.F
    np.testing.assert_allclose(g1[:F * F + fd.E * fd.M + 2 * fd.M], g0[:F * F + fd.E * fd.M + 2 * fd.M], rtol=1e-12,
                               atol=1e-12)


def test_shifted_loss_central_differences():
    """Every shift delta_i, a sample of h pixels and the source positions, central differences
    with a step that stays inside one interpolation cell."""
    fd, P = _field()
    args = (fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W)
    L, _, g, _ = oracle.deconv_loss_grad(*args, P, shifted=True)
    F = fd.F
    od = F * F + fd.E * fd.M + 2 * fd.M
    idx = list(range(od, od + 2 * fd.E)) + [5 * F + 7, 11 * F + 12, 13 * F + 3] + \
        list(range(F * F + fd.E * fd.M, F * F + fd.E * fd.M + 2 * fd.M))
    for j in idx:
        hstep = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[j] += hstep
        Pm[j] -= hstep
        Lp = oracle.deconv_loss_grad(*args, Pp, grad=False, shifted=True)[0]
        Lm = oracle.deconv_loss_grad(*args, Pm, grad=False, shifted=True)[0]
        fdv = (Lp - Lm) / (2 * hstep)
        assert abs(fdv - g[j]) <= 1e-6 * max(abs(g[j]), 1.0) + 1e-6, (j, fdv, g[j])
