"""L-BFGS-B in plain FP64 numpy: the oracle of the library's limited-memory bound-constrained
optimiser (the paper's second optimiser, sec. 2.4).

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module; the product path never
does and shares no code with it.

Written from Byrd, Lu, Nocedal & Zhu (1995), "A limited memory algorithm for bound constrained
optimization", SIAM J. Sci. Comput. 16(5): the compact limited-memory matrix
B = theta I - W M W^T (W = [Y, theta S], M the inverse of [[-D, L^T], [L, theta S^T S]]), the
generalised Cauchy point along the projected steepest-descent path (its breakpoints in increasing
order), the direct primal subspace minimisation over the free variables followed by a backtrack
into the box, and a line search along d = xbar - x.  The line search is the strong-Wolfe
bracketing and zoom of Nocedal & Wright (2006, Algorithms 3.5 and 3.6) with bisection,
c1 = 1e-3, c2 = 0.9, the first step min(1, 1/||d||) at the first iteration and 1 afterwards, never
above 1 (x + d is feasible).  A pair (s, y) enters the memory when s^T y > 2.2e-16 y^T y.
Stopping: projected gradient sup-norm <= pgtol, or (f_k - f_{k+1}) / max(|f_k|, |f_{k+1}|, 1) <=
factr * 2.2e-16, or max_iter iterations, or a failed line search.
"""
from __future__ import annotations

import numpy as np

EPS = 2.220446049250313e-16
C1, C2 = 1e-3, 0.9


def projected_gradient_norm(x, g, lo, hi):
    return float(np.max(np.abs(np.clip(x - g, lo, hi) - x))) if x.size else 0.0


def _middle(S, Y, theta):
    """M of the compact form (2k x 2k) and W = [Y, theta S] (n x 2k); None when k = 0."""
    if not S:
        return None, None
    Sm, Ym = np.stack(S, axis=1), np.stack(Y, axis=1)
    SY = Sm.T @ Ym
    D = np.diag(np.diag(SY))
    L = np.tril(SY, -1)
    K = np.block([[-D, L.T], [L, theta * (Sm.T @ Sm)]])
    return np.hstack([Ym, theta * Sm]), np.linalg.inv(K)


def cauchy_point(x, g, lo, hi, theta, W, M):
    """Generalised Cauchy point (Byrd et al. sec. 4): returns (xc, c, fixed) with c = W^T (xc - x)
    accumulated along the path and `fixed` the variables that reached a bound."""
    n = x.size
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(g < 0, (x - hi) / g, np.where(g > 0, (x - lo) / g, np.inf))
    d = np.where(t == 0.0, 0.0, -g)
    k2 = 0 if W is None else W.shape[1]
    p = W.T @ d if k2 else np.zeros(0)
    c = np.zeros(k2)
    fp = -float(d @ d)
    fpp = -theta * fp - (float(p @ M @ p) if k2 else 0.0)
    fpp0 = -theta * fp
    dtm = -fp / fpp if fpp > 0 else 0.0
    told = 0.0
    xc = x.copy()
    fixed = np.zeros(n, dtype=bool)
    fixed[t == 0.0] = True
    cand = np.where(np.isfinite(t) & (t > 0))[0]
    order = cand[np.argsort(t[cand], kind="stable")]
    for b in order:
        tj = t[b]
        dt = tj - told
        if dtm < dt:
            break
        xcb = hi[b] if d[b] > 0 else lo[b]
        zb = xcb - x[b]
        if k2:
            c = c + dt * p
        gb = g[b]
        fp = fp + dt * fpp + gb * gb + theta * gb * zb
        fpp = fpp - theta * gb * gb
        if k2:
            wb = W[b]
            fp -= gb * float(wb @ M @ c)
            fpp -= 2.0 * gb * float(wb @ M @ p) + gb * gb * float(wb @ M @ wb)
            p = p + gb * wb
        fpp = max(EPS * fpp0, fpp)
        d[b] = 0.0
        xc[b] = xcb
        fixed[b] = True
        dtm = -fp / fpp if fpp > 0 else 0.0
        told = tj
    dtm = max(dtm, 0.0)
    told += dtm
    free_move = ~fixed
    xc[free_move] = x[free_move] + told * d[free_move]
    if k2:
        c = c + dtm * p
    return xc, c, fixed


def subspace_min(x, g, lo, hi, xc, c, fixed, theta, W, M):
    """Direct primal method over the free variables, then the backtrack into the box."""
    free = ~fixed
    if not np.any(free):
        return xc
    k2 = 0 if W is None else W.shape[1]
    rc = g[free] + theta * (xc[free] - x[free])
    if k2:
        rc = rc - W[free] @ (M @ c)
        Wz = W[free]
        v = M @ (Wz.T @ rc)
        Nm = np.eye(k2) - (M @ (Wz.T @ Wz)) / theta
        v = np.linalg.solve(Nm, v)
        du = -rc / theta - (Wz @ v) / (theta * theta)
    else:
        du = -rc / theta
    alpha = 1.0
    xf, lof, hif = xc[free], lo[free], hi[free]
    with np.errstate(divide="ignore", invalid="ignore"):
        lim = np.where(du > 0, (hif - xf) / du, np.where(du < 0, (lof - xf) / du, np.inf))
    if lim.size:
        alpha = min(1.0, float(np.min(lim)))
    xbar = xc.copy()
    xbar[free] = xf + alpha * du
    return xbar


def line_search(fun, x, f0, g0, d, stp0, max_ls=20):
    """Strong Wolfe along d (steps in (0, 1]).  Returns (stp, x, f, g, evaluations) or None."""
    dphi0 = float(g0 @ d)
    if not dphi0 < 0:
        return None
    evals = 0

    def phi(a):
        xa = x + a * d
        fa, ga = fun(xa)
        return xa, fa, ga, float(ga @ d)

    def zoom(a_lo, f_lo, a_hi):
        nonlocal evals
        while evals < max_ls:
            a = 0.5 * (a_lo + a_hi)
            xa, fa, ga, da = phi(a)
            evals += 1
            if fa > f0 + C1 * a * dphi0 or fa >= f_lo:
                a_hi = a
            else:
                if abs(da) <= -C2 * dphi0:
                    return a, xa, fa, ga
                if da * (a_hi - a_lo) >= 0:
                    a_hi = a_lo
                a_lo, f_lo = a, fa
        return None

    a_prev, f_prev = 0.0, f0
    a = stp0
    while evals < max_ls:
        xa, fa, ga, da = phi(a)
        evals += 1
        if fa > f0 + C1 * a * dphi0 or (a_prev > 0 and fa >= f_prev):
            r = zoom(a_prev, f_prev, a)
            return None if r is None else (*r, evals)
        if abs(da) <= -C2 * dphi0:
            return a, xa, fa, ga, evals
        if da >= 0:
            r = zoom(a, fa, a_prev)
            return None if r is None else (*r, evals)
        if a >= 1.0:
            return a, xa, fa, ga, evals  # the whole step is feasible and still descending
        a_prev, f_prev = a, fa
        a = min(2.0 * a, 1.0)
    return None


def lbfgsb(fun, x0, lo, hi, m=10, max_iter=100, pgtol=1e-5, factr=1e7, max_ls=20):
    """Minimise fun (x -> (f, g)) over lo <= x <= hi.  Returns a dict: x, f, g, iterations,
    evaluations, status ('pgtol', 'factr', 'max_iter', 'line_search'), the f of every iterate."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x = np.clip(np.asarray(x0, dtype=np.float64), lo, hi)
    f, g = fun(x)
    evals, S, Y, theta = 1, [], [], 1.0
    hist, status, it = [f], "max_iter", 0
    while it < max_iter:
        if projected_gradient_norm(x, g, lo, hi) <= pgtol:
            status = "pgtol"
            break
        W, M = _middle(S, Y, theta)
        xc, c, fixed = cauchy_point(x, g, lo, hi, theta, W, M)
        xbar = subspace_min(x, g, lo, hi, xc, c, fixed, theta, W, M)
        d = xbar - x
        dn = float(np.linalg.norm(d))
        if dn == 0.0:
            status = "pgtol"
            break
        r = line_search(fun, x, f, g, d, min(1.0, 1.0 / dn) if it == 0 else 1.0, max_ls)
        if r is None:
            status = "line_search"
            break
        _, xn, fn, gn, ne = r
        evals += ne
        s, y = xn - x, gn - g
        if float(s @ y) > EPS * float(y @ y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
            theta = float(y @ y) / float(s @ y)
        fo = f
        x, f, g = xn, fn, gn
        hist.append(f)
        it += 1
        if (fo - f) / max(abs(fo), abs(f), 1.0) <= factr * EPS:
            status = "factr"
            break
    return {"x": x, "f": f, "g": g, "iterations": it, "evaluations": evals, "status": status,
            "history": np.array(hist)}
