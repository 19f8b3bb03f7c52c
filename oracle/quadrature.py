"""Oracle quadrature: collapsed (Stroud conical-product) Gauss-Jacobi rules on simplices.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module; the product path never does.

The action replaces each cell integral by a weighted sum over quadrature points
(the paper's Eq. "poisson_action_w_quadrature"); the paper does not name its rule
(Table "action_param_space" gives only point counts), so the oracle and the
library both use the conical-product rule below, each generated independently.

Rule for exactness degree q on the reference d-simplex {xhat_k >= 0, sum <= 1}:
n = ceil((q+1)/2) Gauss points per direction.  With collapsed coordinates
t in [0,1]^d,

    xhat_1 = t_1,  xhat_2 = t_2 (1 - t_1),  xhat_3 = t_3 (1 - t_1)(1 - t_2),

the Jacobian is (1 - t_1)^{d-1} (1 - t_2)^{d-2} ..., so direction k uses the
Gauss-Jacobi rule for the weight (1 - t)^{d-k} on [0,1].  Points are ordered
with t_1 outermost and t_d innermost, each direction's nodes ascending.

Gauss-Jacobi nodes/weights come from the Golub-Welsch eigenvalue method on the
three-term recurrence of the Jacobi polynomials (weight (1-x)^a (1+x)^b on
[-1,1]), computed with numpy's symmetric eigensolver.
"""

from __future__ import annotations

from math import ceil, gamma

import numpy as np


def gauss_jacobi(n: int, a: float, b: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Jacobi rule for (1-x)^a (1+x)^b on [-1, 1] (Golub-Welsch)."""
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    # diagonal: alpha_k = (b^2 - a^2) / (s (s + 2)); the k=0, a+b=0 limit is (b-a)/(a+b+2)
    with np.errstate(divide="ignore", invalid="ignore"):
        diag = (b * b - a * a) / (s * (s + 2.0))
    if abs(a + b) < 1e-300:
        diag[0] = (b - a) / (a + b + 2.0)
    # off-diagonal: beta_k for k = 1..n-1
    kk = np.arange(1, n, dtype=np.float64)
    ss = 2.0 * kk + a + b
    beta = 4.0 * kk * (kk + a) * (kk + b) * (kk + a + b) / (ss * ss * (ss + 1.0) * (ss - 1.0))
    T = np.diag(diag) + np.diag(np.sqrt(beta), 1) + np.diag(np.sqrt(beta), -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + b + 1.0) * gamma(a + 1.0) * gamma(b + 1.0) / gamma(a + b + 2.0)
    w = mu0 * V[0, :] ** 2
    order = np.argsort(x)
    return x[order], w[order]


def gauss_jacobi_01(n: int, a: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point rule for the weight (1-t)^a on [0, 1]."""
    x, w = gauss_jacobi(n, float(a), 0.0)
    t = 0.5 * (1.0 + x)
    # int_0^1 f(t) (1-t)^a dt = 2^{-a-1} int_{-1}^{1} f((1+x)/2) (1-x)^a dx
    return t, w * 2.0 ** (-a - 1.0)


def points_per_direction(quad_degree: int) -> int:
    return int(ceil((quad_degree + 1) / 2))


def simplex_rule(dim: int, quad_degree: int) -> tuple[np.ndarray, np.ndarray]:
    """Conical-product rule exact to ``quad_degree``: points [Q, dim], weights [Q]."""
    if dim not in (1, 2, 3):
        raise ValueError("dim in 1..3")
    if quad_degree < 0:
        raise ValueError("quad_degree >= 0")
    n = points_per_direction(quad_degree)
    rules = [gauss_jacobi_01(n, dim - 1 - k) for k in range(dim)]  # direction k+1
    pts, wts = [], []

    def rec(k, t, w):
        if k == dim:
            x = np.zeros(dim)
            scale = 1.0
            for m in range(dim):
                x[m] = t[m] * scale
                scale *= (1.0 - t[m])
            pts.append(x)
            wts.append(w)
            return
        tk, wk = rules[k]
        for i in range(n):
            rec(k + 1, t + [tk[i]], w * wk[i])

    rec(0, [], 1.0)
    return np.asarray(pts), np.asarray(wts)
