"""Oracle Lagrange basis on the reference simplex and its tabulation.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module; the product path never does.

The tabulation matrices Phi_k[q, j] are the reference basis functions (k = 0)
and their reference partial derivatives (k = 1..d) at the quadrature points
(the paper's Eq. "poisson_tabulated_values"; Algorithm 2 reads them in its
evaluation and quadrature phases).

Basis: equispaced P_p Lagrange functions written with Silvester's barycentric
product formula.  For node multi-index alpha (alpha_0 = p - sum alpha_k) and
barycentric coordinates lam_0 = 1 - sum xhat_k, lam_k = xhat_k,

    phi_alpha(lam) = prod_{m=0..d} prod_{i=0..alpha_m - 1} (p lam_m - i) / (i + 1).

Derivatives use the product rule with d lam_0 / d xhat_k = -1 and
d lam_m / d xhat_k = delta_mk.  Local node order: multi-indices
(alpha_1..alpha_d), alpha_1 outermost and alpha_d innermost in nested ascending
loops (this order is an interface convention with the mesh's cell2node).
"""

from __future__ import annotations

import numpy as np

from .quadrature import simplex_rule


def multi_indices(dim: int, degree: int) -> list[tuple[int, ...]]:
    out: list[tuple[int, ...]] = []

    def rec(prefix, remaining):
        if len(prefix) == dim:
            out.append(tuple(prefix))
            return
        for a in range(remaining + 1):
            rec(prefix + [a], remaining - a)

    rec([], degree)
    return out


def _factor(p: int, a: int, lam: float) -> tuple[float, float]:
    """prod_{i<a} (p lam - i)/(i+1) and its derivative with respect to lam."""
    val = 1.0
    der = 0.0
    for i in range(a):
        f = (p * lam - i) / (i + 1.0)
        df = p / (i + 1.0)
        der = der * f + val * df
        val = val * f
    return val, der


def basis_at(dim: int, degree: int, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Values [n] and reference gradients [d, n] of all basis functions at point x."""
    alphas = multi_indices(dim, degree)
    lam = np.empty(dim + 1)
    lam[0] = 1.0 - float(np.sum(x))
    lam[1:] = x
    # d lam_m / d xhat_k
    dlam = np.zeros((dim + 1, dim))
    dlam[0, :] = -1.0
    for k in range(dim):
        dlam[k + 1, k] = 1.0
    n = len(alphas)
    val = np.empty(n)
    grad = np.zeros((dim, n))
    for j, al in enumerate(alphas):
        full = (degree - sum(al),) + tuple(al)
        f = [_factor(degree, full[m], lam[m]) for m in range(dim + 1)]
        v = 1.0
        for m in range(dim + 1):
            v *= f[m][0]
        val[j] = v
        for m in range(dim + 1):
            # derivative of factor m times the other factors
            other = 1.0
            for mm in range(dim + 1):
                if mm != m:
                    other *= f[mm][0]
            for k in range(dim):
                grad[k, j] += f[m][1] * dlam[m, k] * other
    return val, grad


def tabulate(dim: int, degree: int, quad_degree: int, scheme: str = "conical"):
    """(points [Q,d], weights [Q], tab [1+d, Q, n]) for the oracle's own rule
    (``scheme``: "conical" product rule or "symmetric" rule family)."""
    if scheme == "symmetric":
        from .symmetric import symmetric_rule
        pts, wts = symmetric_rule(dim, quad_degree)
    else:
        pts, wts = simplex_rule(dim, quad_degree)
    n = len(multi_indices(dim, degree))
    tab = np.empty((1 + dim, len(wts), n))
    for q in range(len(wts)):
        v, g = basis_at(dim, degree, pts[q])
        tab[0, q, :] = v
        tab[1:, q, :] = g
    return pts, wts, tab
