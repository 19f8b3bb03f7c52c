"""Oracle: fully symmetric quadrature rules on triangles and tetrahedra.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module.

A fully symmetric rule is invariant under every permutation of the barycentric
coordinates; its points form orbits sharing one weight.  Given an orbit
structure (centroid; (a,a,1-2a) and (a,b,1-a-b) on triangles; (a,a,a,1-3a),
(a,a,1/2-a,1/2-a), (a,a,b,1-2a-b) on tetrahedra) the rule is the solution of the
moment equations sum_i w_i xhat_i^alpha = alpha!/(|alpha|+d)! for |alpha| <= q,
found here with scipy.optimize.least_squares (each equation relative to its
right-hand side) from a rough starting point, polished by Gauss-Newton steps in
numpy longdouble (extended precision) and rounded once, and accepted only with
positive weights, interior points and relative residual < 1e-13.  The
family selected for a requested degree q is the tabulated rule of the smallest
degree >= q, else the conical-product rule.  Points are sorted lexicographically.
"""

from __future__ import annotations

import itertools
from math import factorial

import numpy as np
from scipy.optimize import least_squares

from .quadrature import simplex_rule

# (dim, degree) -> (orbit kinds, rough start: per orbit parameters then the
# weight of each point of the orbit)
RULES = {
    (2, 2): (["S21"], [0.17, 0.17]),
    (2, 4): (["S21", "S21"], [0.446, 0.0372, 0.0916, 0.0183]),
    (2, 6): (["S21", "S21", "S111"], [0.249, 0.0195, 0.0631, 0.00847, 0.0531, 0.310, 0.0069]),
    (2, 8): (["S3", "S21", "S21", "S21", "S111"],
             [0.0722, 0.459, 0.0159, 0.171, 0.0172, 0.0505, 0.00541, 0.00839, 0.263, 0.00227]),
    (3, 2): (["S31"], [0.138, 0.0417]),
    (3, 5): (["S31", "S31", "S22"], [0.311, 0.0188, 0.0927, 0.0122, 0.0455, 0.00709]),
    # degree 6, 24 points (Keast's orbit structure: three S31 orbits and one S211)
    (3, 6): (["S31", "S31", "S31", "S211"],
             [0.215, 0.00665, 0.0407, 0.00168, 0.322, 0.00923, 0.0637, 0.270, 0.00804]),
}
NPAR = {"S3": 0, "S4": 0, "S21": 1, "S31": 1, "S22": 1, "S111": 2, "S211": 2}


def _points(kinds, x, dtype=np.float64):
    pts, wts, i = [], [], 0
    one = dtype(1)
    for kind in kinds:
        k = NPAR[kind]
        par, w = x[i:i + k], x[i + k]
        i += k + 1
        if kind == "S3":
            lam = (one / 3,) * 3
        elif kind == "S21":
            lam = (par[0], par[0], one - 2 * par[0])
        elif kind == "S111":
            lam = (par[0], par[1], one - par[0] - par[1])
        elif kind == "S4":
            lam = (one / 4,) * 4
        elif kind == "S31":
            lam = (par[0],) * 3 + (one - 3 * par[0],)
        elif kind == "S22":
            lam = (par[0], par[0], one / 2 - par[0], one / 2 - par[0])
        else:  # S211
            lam = (par[0], par[0], par[1], one - 2 * par[0] - par[1])
        seen = set()
        for perm in itertools.permutations(lam):
            key = tuple(float(v) for v in perm)
            if key in seen:
                continue
            seen.add(key)
            pts.append(perm[1:])
            wts.append(w)
    return np.array(pts, dtype=dtype), np.array(wts, dtype=dtype)


def _moments(dim, q, dtype=np.float64):
    out = []
    for alpha in itertools.product(range(q + 1), repeat=dim):
        if sum(alpha) <= q:
            num = 1
            for a in alpha:
                num *= factorial(a)
            out.append((np.array(alpha), dtype(num) / dtype(factorial(sum(alpha) + dim))))
    return out


def _residual(kinds, dim, q, x, dtype):
    pts, wts = _points(kinds, x, dtype)
    # relative residual per moment (high-degree moments are small)
    return np.array([np.sum(wts * np.prod(pts ** a, axis=1)) / v - dtype(1)
                     for a, v in _moments(dim, q, dtype)], dtype=dtype)


def _gauss_newton_ext(kinds, dim, q, x, iters=40):
    """Gauss-Newton in numpy longdouble (extended precision) with its own
    elimination; keeps the best iterate."""
    L = np.longdouble
    x = np.array(x, dtype=L)
    best_x, best_r = x.copy(), np.abs(_residual(kinds, dim, q, x, L)).max()
    for _ in range(iters):
        r = _residual(kinds, dim, q, x, L)
        n = len(x)
        J = np.empty((len(r), n), dtype=L)
        for j in range(n):
            h = L(1e-9) * max(L(1), abs(x[j]))
            e = np.zeros(n, dtype=L)
            e[j] = h
            J[:, j] = (_residual(kinds, dim, q, x + e, L) - _residual(kinds, dim, q, x - e, L)) / (2 * h)
        A = J.T @ J
        g = -(J.T @ r)
        M = np.concatenate([A, g[:, None]], axis=1)
        for c in range(n):                       # elimination with partial pivoting
            piv = c + int(np.argmax(np.abs(M[c:, c])))
            M[[c, piv]] = M[[piv, c]]
            for k in range(c + 1, n):
                M[k] -= M[k, c] / M[c, c] * M[c]
        dx = np.zeros(n, dtype=L)
        for c in range(n - 1, -1, -1):
            dx[c] = (M[c, n] - M[c, c + 1:n] @ dx[c + 1:]) / M[c, c]
        x = x + dx
        rx = np.abs(_residual(kinds, dim, q, x, L)).max()
        if rx < best_r:
            best_x, best_r = x.copy(), rx
    return best_x, best_r


def _solve(dim, degree):
    kinds, x0 = RULES[(dim, degree)]
    sol = least_squares(lambda x: _residual(kinds, dim, degree, x, np.float64),
                        np.array(x0, float), xtol=3e-16, ftol=3e-16, gtol=3e-16, max_nfev=2000)
    xl, rl = _gauss_newton_ext(kinds, dim, degree, sol.x)
    x = xl.astype(np.float64)        # round once
    pts, wts = _points(kinds, x)
    if not (rl < 1e-13 and np.all(wts > 0) and np.all(pts > 0) and np.all(pts.sum(axis=1) < 1)):
        raise RuntimeError(f"symmetric rule {(dim, degree)} did not converge")
    order = np.lexsort(pts.T[::-1])
    return pts[order], wts[order]


def symmetric_rule(dim: int, quad_degree: int):
    """(points [Q, dim], weights [Q]) of the rule family selected for quad_degree."""
    degs = sorted(d for (dd, d) in RULES if dd == dim and d >= quad_degree)
    if not degs:
        return simplex_rule(dim, quad_degree)
    return _solve(dim, degs[0])
