"""Pins for the paper's accuracy metrics (sec. 3): closed forms of each definition."""
import numpy as np
import pytest

from paper_2402_08725_gb300 import metrics as mt


def test_p_astro_removes_the_common_bias():
    c = np.array([[0.0, 0.0], [3.0, -1.0], [-2.0, 4.0]])
    assert mt.p_astro(c, c) == 0.0
    assert mt.p_astro(c, c + np.array([0.3, -0.2])) == pytest.approx(0.0, abs=1e-15)  # a pure offset is bias
    np.testing.assert_allclose(mt.astrometric_bias(c, c + np.array([0.3, -0.2])), [-0.3, 0.2])
    # two positions with opposite errors +-e: no bias, each off by |e|
    e = np.array([0.3, 0.4])
    est = c[:2] + np.array([e, -e])
    assert mt.p_astro(c[:2], est) == pytest.approx(0.5)
    assert mt.p_astro(c[:1], c[:1] + e) == 0.0  # one position: all of its error is bias


def test_photometric_accuracy_and_precision():
    f = np.array([100.0, 250.0, 40.0, 1e4])
    assert mt.a_photo(f, f) == 0.0 and mt.p_photo(f, f) == 0.0
    eps = 0.05
    est = f / (1.0 + eps)  # every estimate low by the same factor: relative error eps, no scatter
    assert mt.a_photo(f, est) == pytest.approx(eps)
    assert mt.p_photo(f, est) == pytest.approx(0.0, abs=1e-15)
    # errors +-r relative to the estimates: accuracy 0, precision r
    est = np.array([100.0, 250.0, 40.0, 1e4])
    tru = est * np.array([1.1, 0.9, 1.1, 0.9])
    assert mt.a_photo(tru, est) == pytest.approx(0.0, abs=1e-15)
    assert mt.p_photo(tru, est) == pytest.approx(0.1)
    # the mask keeps the selected entries only
    assert mt.a_photo(tru, est, mask=[True, False, True, False]) == pytest.approx(0.1)


def test_mae_psf_is_the_l1_distance():
    rng = np.random.default_rng(0)
    p = rng.random((9, 9))
    q = p.copy()
    q[4, 4] += 0.25
    q[0, 1] -= 0.5
    assert mt.mae_psf(p, q) == pytest.approx(0.75)
    assert mt.mae_psf(p, p) == 0.0
