"""Exact rational element matrices on simplices (pins the oracle without quadrature).

Polynomials are dicts {barycentric exponent tuple: Fraction}.  Integrals use the
closed form int_T lam^beta dx = d! |T| beta! / (|beta| + d)!, so no quadrature
rule, tabulation or floating point enters.  The Lagrange basis is Silvester's
product formula expanded symbolically; gradients use the constant barycentric
gradients of the (rational) cell.
"""

from __future__ import annotations

from fractions import Fraction
from math import factorial


def _mul(p, q):
    out = {}
    for a, ca in p.items():
        for b, cb in q.items():
            k = tuple(x + y for x, y in zip(a, b))
            out[k] = out.get(k, 0) + ca * cb
    return {k: v for k, v in out.items() if v != 0}


def _add(p, q, s=1):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, 0) + s * v
    return {k: v for k, v in out.items() if v != 0}


def _scale(p, s):
    return {k: v * s for k, v in p.items() if v * s != 0}


def _diff(p, m):
    """d/d lam_m."""
    out = {}
    for k, v in p.items():
        if k[m] > 0:
            kk = list(k)
            kk[m] -= 1
            out[tuple(kk)] = out.get(tuple(kk), 0) + v * k[m]
    return out


def multi_indices(dim, degree):
    out = []

    def rec(prefix, remaining):
        if len(prefix) == dim:
            out.append(tuple(prefix))
            return
        for a in range(remaining + 1):
            rec(prefix + [a], remaining - a)

    rec([], degree)
    return out


def lagrange_basis(dim, degree):
    """Symbolic basis polynomials in (lam_0..lam_d), in the documented node order."""
    basis = []
    for al in multi_indices(dim, degree):
        full = (degree - sum(al),) + tuple(al)
        poly = {(0,) * (dim + 1): Fraction(1)}
        for m in range(dim + 1):
            for i in range(full[m]):
                e = [0] * (dim + 1)
                e[m] = 1
                lin = {tuple(e): Fraction(degree, i + 1)}
                if i:
                    lin[(0,) * (dim + 1)] = Fraction(-i, i + 1)
                poly = _mul(poly, lin)
        basis.append(poly)
    return basis


def _det(M):
    n = len(M)
    if n == 1:
        return M[0][0]
    return sum((-1) ** j * M[0][j] * _det([row[:j] + row[j + 1:] for row in M[1:]]) for j in range(n))


def _inv(M):
    n = len(M)
    A = [list(map(Fraction, row)) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [x / piv for x in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [row[n:] for row in A]


class ExactCell:
    def __init__(self, X):
        """X: list of d+1 vertices with Fraction coordinates."""
        self.d = len(X) - 1
        d = self.d
        X = [[Fraction(c) for c in v] for v in X]
        J = [[X[k + 1][i] - X[0][i] for k in range(d)] for i in range(d)]
        self.vol = abs(_det(J)) / factorial(d)
        # lam = B^{-1} [1; x]  with B = [[1..1]; [x_0 .. x_d]]
        B = [[Fraction(1)] * (d + 1)] + [[X[m][i] for m in range(d + 1)] for i in range(d)]
        Binv = _inv(B)
        self.dlam = [[Binv[m][i + 1] for i in range(d)] for m in range(d + 1)]  # d lam_m / dx_i

    def integrate(self, p):
        d = self.d
        s = Fraction(0)
        for beta, c in p.items():
            num = factorial(d) * self.vol
            for b in beta:
                num *= factorial(b)
            s += c * num / factorial(sum(beta) + d)
        return s

    def grad(self, p):
        return [
            {k: v for k, v in _sum_terms([_scale(_diff(p, m), self.dlam[m][i]) for m in range(self.d + 1)]).items()}
            for i in range(self.d)]


def _sum_terms(terms):
    out = {}
    for t in terms:
        out = _add(out, t)
    return out


def element_mass(X, degree):
    cell = ExactCell(X)
    B = lagrange_basis(cell.d, degree)
    n = len(B)
    return [[cell.integrate(_mul(B[i], B[j])) for j in range(n)] for i in range(n)]


def element_elasticity(X, degree, lam, mu):
    """K[(i,a),(j,b)] = int lam d_b phi_j d_a phi_i + mu delta_ab grad phi_j . grad phi_i
    + mu d_a phi_j d_b phi_i   (sigma(phi_j e_b) : grad(phi_i e_a))."""
    cell = ExactCell(X)
    d = cell.d
    lam, mu = Fraction(lam), Fraction(mu)
    B = lagrange_basis(d, degree)
    n = len(B)
    G = [cell.grad(b) for b in B]
    prod = {}

    def I(i, a, j, b):
        key = (i, a, j, b)
        if key not in prod:
            prod[key] = cell.integrate(_mul(G[i][a], G[j][b]))
        return prod[key]

    K = [[Fraction(0)] * (n * d) for _ in range(n * d)]
    for i in range(n):
        for a in range(d):
            for j in range(n):
                for b in range(d):
                    v = lam * I(j, b, i, a) + mu * I(j, a, i, b)
                    if a == b:
                        v += mu * sum(I(j, k, i, k) for k in range(d))
                    K[i * d + a][j * d + b] = v
    return K


def element_laplace(X, degree):
    """K[i][j] = int grad phi_i . grad phi_j."""
    cell = ExactCell(X)
    d = cell.d
    B = lagrange_basis(d, degree)
    G = [cell.grad(b) for b in B]
    n = len(B)
    return [[sum(cell.integrate(_mul(G[i][k], G[j][k])) for k in range(d)) for j in range(n)]
            for i in range(n)]


def assemble(cells_X, cell2node, n_nodes, degree, kind, ncomp=1, **kw):
    """Exact global matrix from element matrices (Fractions)."""
    N = n_nodes * ncomp
    A = [[Fraction(0)] * N for _ in range(N)]
    for X, nodes in zip(cells_X, cell2node):
        if kind == "mass":
            Ke = element_mass(X, degree)
        elif kind == "laplace":
            Ke = element_laplace(X, degree)
        elif kind == "helmholtz":
            Kl, Km = element_laplace(X, degree), element_mass(X, degree)
            Ke = [[a + b for a, b in zip(ra, rb)] for ra, rb in zip(Kl, Km)]
        else:
            Ke = element_elasticity(X, degree, kw["lam"], kw["mu"])
        dofs = [int(nd) * ncomp + c for nd in nodes for c in range(ncomp)]
        for r, gr in enumerate(dofs):
            for s, gs in enumerate(dofs):
                A[gr][gs] += Ke[r][s]
    return A
