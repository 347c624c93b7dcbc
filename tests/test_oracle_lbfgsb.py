"""Pins for the oracle's L-BFGS-B (Byrd, Lu, Nocedal & Zhu 1995): exact minimisers of bounded
strictly convex quadratics found by enumerating every active set, the reference L-BFGS-B of
scipy on bounded Rosenbrock problems, and the unconstrained minimiser of a quadratic."""
import itertools

import numpy as np
import pytest
import scipy.optimize

from oracle import lbfgsb as lb


def _qp_exact(A, b, lo, hi):
    """min 1/2 x^T A x - b^T x on the box by brute force: every (lower, upper, free) pattern,
    the KKT point of the pattern kept when it is feasible with multipliers of the right sign."""
    n = b.size
    best = None
    for pat in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pat)
        x = np.where(pat == 0, lo, np.where(pat == 1, hi, 0.0))
        fr = pat == 2
        if fr.any():
            rhs = b[fr] - A[np.ix_(fr, ~fr)] @ x[~fr]
            x[fr] = np.linalg.solve(A[np.ix_(fr, fr)], rhs)
        if np.any(x < lo - 1e-12) or np.any(x > hi + 1e-12):
            continue
        g = A @ x - b
        if np.any(g[pat == 0] < -1e-10) or np.any(g[pat == 1] > 1e-10):
            continue
        val = 0.5 * x @ A @ x - b @ x
        if best is None or val < best[1]:
            best = (x, val)
    return best[0]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bounded_quadratic_matches_active_set_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = 6
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + 0.5 * np.eye(n)
    b = rng.normal(scale=3.0, size=n)
    lo = np.where(rng.random(n) < 0.7, -0.5, -np.inf)
    hi = np.where(rng.random(n) < 0.5, 0.4, np.inf)
    ref = _qp_exact(A, b, np.where(np.isinf(lo), -1e30, lo), np.where(np.isinf(hi), 1e30, hi))
    res = lb.lbfgsb(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(n), lo, hi, pgtol=1e-10,
                    factr=1.0, max_iter=500)
    np.testing.assert_allclose(res["x"], ref, atol=1e-7)
    assert np.all(res["x"] >= lo) and np.all(res["x"] <= hi)


def _rosen(x):
    return scipy.optimize.rosen(x), scipy.optimize.rosen_der(x)


@pytest.mark.parametrize("n,lo_v,hi_v", [(2, -2.0, 0.8), (5, -1.5, 0.9), (10, 0.2, 2.0)])
def test_bounded_rosenbrock_matches_scipy(n, lo_v, hi_v):
    x0 = np.full(n, -1.0 if lo_v < 0 else 1.5)
    lo, hi = np.full(n, lo_v), np.full(n, hi_v)
    res = lb.lbfgsb(_rosen, x0, lo, hi, pgtol=1e-9, factr=10.0, max_iter=2000)
    ref = scipy.optimize.minimize(_rosen, x0, jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                                  options={"gtol": 1e-10, "ftol": 1e-15, "maxiter": 5000})
    np.testing.assert_allclose(res["x"], ref.x, atol=2e-5)
    assert res["f"] <= ref.fun + 1e-9


def test_unconstrained_quadratic():
    rng = np.random.default_rng(9)
    n = 30
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + np.eye(n)
    b = rng.normal(size=n)
    inf = np.full(n, np.inf)
    res = lb.lbfgsb(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(n), -inf, inf, pgtol=1e-10,
                    factr=1.0, max_iter=1000)
    np.testing.assert_allclose(res["x"], np.linalg.solve(A, b), atol=1e-7)


def test_first_cauchy_point_on_a_separable_quadratic():
    """f = 1/2 |x|^2 - b.x with B = I: the generalised Cauchy point of the first iteration is the
    projection of x - 1 * g (the path's model minimum lies at t = 1 when no breakpoint comes
    first), i.e. clip(b, lo, hi) for x = 0."""
    b = np.array([2.0, -1.0, 0.3, -3.0])
    lo, hi = np.array([-np.inf, -0.5, 0.0, -1.0]), np.array([1.0, np.inf, np.inf, 0.0])
    x = np.zeros(4)
    xc, _, fixed = lb.cauchy_point(x, x - b, lo, hi, 1.0, None, None)
    np.testing.assert_allclose(xc, np.clip(b, lo, hi))
    assert list(fixed) == [True, True, False, True]
