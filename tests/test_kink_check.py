"""The parity helper's handling of the starlet prior's kinks (reading R14), on the CPU: a
subgradient that differs from the oracle's only at coefficients FP32 cannot decide is accepted,
and an error anywhere else is still caught."""
import numpy as np

import oracle
from paper_2402_08725_gb300 import synthetic as syn
from tests._helpers import GRAD_RTOL, check_h_with_kinks, prior_kinks, rel_l2


def _field_and_prior_grads():
    # a 32x32 config-4-like field whose h has one finest-scale coefficient within FP32 rounding of 0
    fd = syn.config4_field(4, 32, 12, 4)
    F, J = fd.F, fd.J
    h = fd.params[:F * F].astype(np.float64).reshape(F, F)
    planes = oracle.starlet_analysis(h, J)
    sg = np.sign(planes)
    sg[-1] = 0.0
    for j in range(J - 1):
        sg[j] *= fd.lam * fd.W[j]
    return fd, h, planes, sg


def test_sign_choice_at_an_undecidable_coefficient_is_accepted():
    fd, h, planes, sg = _field_and_prior_grads()
    n, allow = prior_kinks(h, fd.J, fd.lam, fd.W)
    assert n >= 1
    # the undecidable coefficient: the finest-plane one closest to zero relative to |h| around it
    ratio = np.abs(planes[0]) / np.maximum(np.abs(h), 1e-30)
    y, x = np.unravel_index(np.argmin(ratio), ratio.shape)
    assert allow[y, x] > 0.0
    g_ref = oracle.starlet_adjoint(sg).ravel()
    for flipped in (0.0, -sg[0, y, x]):   # the GPU may take sign 0 or the opposite sign there
        sg2 = sg.copy()
        sg2[0, y, x] = flipped
        g = oracle.starlet_adjoint(sg2).ravel()
        assert rel_l2(g, g_ref) > GRAD_RTOL   # the plain check alone would reject it
        res = {}
        assert check_h_with_kinks(fd, g, g_ref, fd.params, res), res


def test_errors_away_from_kinks_still_fail():
    fd, h, planes, sg = _field_and_prior_grads()
    F = fd.F
    _, allow = prior_kinks(h, fd.J, fd.lam, fd.W)
    g_ref = oracle.starlet_adjoint(sg).ravel()
    ys, xs = np.nonzero(allow == 0.0)
    k = len(ys) // 2
    g_bad = g_ref.copy()
    g_bad[ys[k] * F + xs[k]] += 0.05 * np.abs(g_ref).max() + 1.0
    assert rel_l2(g_bad, g_ref) > GRAD_RTOL
    res = {}
    assert not check_h_with_kinks(fd, g_bad, g_ref, fd.params, res), res
