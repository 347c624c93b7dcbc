"""Shared comparison helpers of the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (stated per result): loss within 1e-6 relative to the oracle's loss L itself;
gradient within 1e-4 relative L2 per parameter block.  Only evaluations at (or next to) a
noiseless truth, where L is close to zero and a relative bound on L is meaningless, are
called with near_zero=True: their loss error is measured against max(L, 1e-3 * 0.5 * sum w d^2)
instead.  Every report carries both ratios ("loss_rel_L" against L, "loss_rel" the one
asserted) and says whether the floor applied ("floor").
"""
import numpy as np

import oracle

LOSS_RTOL = 1e-6
GRAD_RTOL = 1e-4

DECONV_BLOCKS = ("h", "a", "c", "delta", "Gamma")
PSF_BLOCKS = ("b", "moffat", "a", "c")


def loss_scale(L_ref, d, sigma):
    d = np.asarray(d, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    w = np.where(np.isinf(s), 0.0, 1.0 / (s * s))
    return max(abs(L_ref), 1e-3 * 0.5 * float(np.sum(w * d * d)))


def deconv_blocks(E, N, f, M):
    F = f * N
    sizes = [F * F, E * M, 2 * M, 2 * E, E]
    out, o = {}, 0
    for name, n in zip(DECONV_BLOCKS, sizes):
        out[name] = slice(o, o + n)
        o += n
    return out


def psf_blocks(S, N, f):
    F = f * N
    sizes = [F * F, 2, S, 2 * S]
    out, o = {}, 0
    for name, n in zip(PSF_BLOCKS, sizes):
        out[name] = slice(o, o + n)
        o += n
    return out


def rel_l2(g, ref):
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nr = np.linalg.norm(ref)
    if nr == 0.0:
        return float(np.linalg.norm(g))
    return float(np.linalg.norm(g - ref) / nr)


def oracle_deconv(fd, params=None, **kw):
    P = fd.params if params is None else params
    return oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W, P, **kw)


EPS32 = 2.0 ** -24


def _box_count(mask, r):
    """Number of True entries of mask within the (2r+1) x (2r+1) box around each entry."""
    F = mask.shape[0]
    c = np.zeros((F + 1, F + 1))
    c[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.float64), axis=0), axis=1)
    lo = np.clip(np.arange(F) - r, 0, F)
    hi = np.clip(np.arange(F) + r + 1, 0, F)
    return c[hi][:, hi] - c[lo][:, hi] - c[hi][:, lo] + c[lo][:, lo]


def prior_kinks(h, J, lam, W, safety=16.0):
    """Starlet coefficients of h whose sign FP32 arithmetic cannot decide (reading R14: the L1
    subgradient jumps at 0), and the most the prior's subgradient can differ because of them at
    each fine pixel.

    The FP32 kernels compute detail plane j with a rounding error of about j eps32 (|c|_{j-1} +
    |c|_j), |c| the same smoothings of |h| (the B3 filter is non-negative).  A coefficient of the
    FP64 oracle within `safety` times that of zero may take either sign, or 0, on the GPU.  Such a
    choice moves dL/dh by at most 2 lam W_j |A^T e_(j,u)| <= 2 lam W_j, only within the support of
    that atom (radius 2 (2^j - 1) fine pixels).  Returns (count, allowance per pixel)."""
    F = h.shape[0]
    planes = oracle.starlet_analysis(h, J)
    pabs = oracle.starlet_analysis(np.abs(h), J)
    cabs_prev = np.abs(h)
    allow = np.zeros((F, F))
    n = 0
    for j in range(1, J):
        cabs = cabs_prev - pabs[j - 1]
        bound = safety * j * EPS32 * (np.abs(cabs_prev) + np.abs(cabs))
        amb = (np.abs(planes[j - 1]) <= bound) & (bound > 0)
        k = int(amb.sum())
        if k:
            n += k
            Wj = np.asarray(W, dtype=np.float64)[j - 1]
            allow += 2.0 * lam * float(np.max(Wj)) * _box_count(amb, 2 * (2 ** j - 1))
        cabs_prev = cabs
    return n, allow


def check_h_with_kinks(fd, g_h, gref_h, P, res):
    """The h block when its plain rel-L2 fails: outside the footprints of the undecidable
    coefficients (prior_kinks) within GRAD_RTOL; inside them within the allowance."""
    F = fd.F
    h = np.asarray(P[:F * F], dtype=np.float64).reshape(F, F)
    n, allow = prior_kinks(h, fd.J, fd.lam, fd.W)
    diff = (np.asarray(g_h, dtype=np.float64) - gref_h).reshape(F, F)
    mask = allow > 0
    nr = np.linalg.norm(gref_h)
    out = float(np.linalg.norm(diff[~mask]) / nr) if nr > 0 else 0.0
    slack = GRAD_RTOL * float(np.abs(gref_h).max())
    inside = bool(np.all(np.abs(diff[mask]) <= allow[mask] + slack))
    res.update({"h_kinks": n, "h_outside_kinks": out, "h_kink_pixels": int(mask.sum()), "h_inside_ok": inside})
    return out <= GRAD_RTOL and inside


def loss_errors(loss, L_ref, d, sigma, near_zero):
    """(asserted ratio, ratio against L itself, floor used) of a loss against the oracle's."""
    rel_L = abs(loss - L_ref) / abs(L_ref) if L_ref != 0.0 else abs(loss)
    if not near_zero:
        return rel_L, rel_L, False
    scale = loss_scale(L_ref, d, sigma)
    return abs(loss - L_ref) / scale, rel_L, scale > abs(L_ref)


def check_deconv(fd, loss, grad, params=None, report=None, lam_pts=0.0, near_zero=False, shifted=False, theta=None):
    """lam_pts > 0 adds the point-source prior of Eq. 11 to the reference; near_zero=True for
    evaluations at a noiseless truth (see the module docstring); shifted=True takes the oracle
    whose extended channel moves with each epoch's shift, theta the one with rotated frames."""
    L_ref, _, g_ref, _ = oracle_deconv(fd, params, shifted=shifted, theta=theta)
    if lam_pts > 0.0:
        P = fd.params if params is None else params
        v, gp = oracle.pts_prior(fd.E, fd.N, fd.f, fd.M, fd.J, lam_pts, fd.W, P)
        L_ref += v
        g_ref = g_ref + gp
    err, rel_L, floor = loss_errors(loss, L_ref, fd.d, fd.sigma, near_zero)
    res = {"loss": loss, "loss_ref": L_ref, "loss_rel": err, "loss_rel_L": rel_L, "floor": floor}
    g = np.asarray(grad, dtype=np.float64)
    for name, sl in deconv_blocks(fd.E, fd.N, fd.f, fd.M).items():
        if sl.stop > sl.start:
            res[name] = rel_l2(g[sl], g_ref[sl])
    if report is not None:
        report.update(res)
    assert err <= LOSS_RTOL, res
    h_ok = res["h"] <= GRAD_RTOL
    if not h_ok and fd.lam > 0 and lam_pts == 0.0:
        F = fd.F
        h_ok = check_h_with_kinks(fd, g[:F * F], g_ref[:F * F], fd.params if params is None else params, res)
    assert h_ok, ("h", res)
    for name in DECONV_BLOCKS[1:]:
        if name in res:
            assert res[name] <= GRAD_RTOL, (name, res)
    return res


def check_psf(pb, loss, grad, params=None, near_zero=False):
    P = pb.params if params is None else params
    L_ref, _, g_ref = oracle.psf_loss_grad(pb.S, pb.N, pb.f, pb.J, pb.lam, pb.t, pb.sigma, pb.W, P)
    err, rel_L, floor = loss_errors(loss, L_ref, pb.t, pb.sigma, near_zero)
    res = {"loss": loss, "loss_ref": L_ref, "loss_rel": err, "loss_rel_L": rel_L, "floor": floor}
    g = np.asarray(grad, dtype=np.float64)
    for name, sl in psf_blocks(pb.S, pb.N, pb.f).items():
        res[name] = rel_l2(g[sl], g_ref[sl])
    assert err <= LOSS_RTOL, res
    for name in PSF_BLOCKS:
        assert res[name] <= GRAD_RTOL, (name, res)
    return res
