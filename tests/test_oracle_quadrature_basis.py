"""Pins for the oracle's quadrature and tabulation (no GPU).

Quadrature: the rule replaces the cell integral by a weighted sum (Eq.
"poisson_action_w_quadrature"); pinned by exactness on every monomial up to the
rule's degree against the closed form int_That xhat^a = prod a_k! / (|a| + d)!,
and its 1D building block against scipy's Gauss-Jacobi routine.
Basis/tabulation (Eq. "poisson_tabulated_values"): nodality, partition of
unity, zero gradient sum, reproduction of P_p, central differences of values.
"""

import itertools
import json
import os
from math import comb, factorial

import numpy as np
import pytest
import scipy.special

from oracle import basis, quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def monomial_integral(alpha):
    num = 1
    for a in alpha:
        num *= factorial(a)
    return num / factorial(sum(alpha) + len(alpha))


@pytest.mark.parametrize("n,a", [(1, 0), (3, 0), (5, 1), (4, 2), (7, 2), (9, 1)])
def test_gauss_jacobi_matches_scipy(n, a):
    x, w = quadrature.gauss_jacobi(n, float(a), 0.0)
    xs, ws = scipy.special.roots_jacobi(n, float(a), 0.0)
    order = np.argsort(xs)
    np.testing.assert_allclose(x, xs[order], rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, ws[order], rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("q", [0, 1, 2, 3, 4, 6, 8, 12])
def test_simplex_rule_exact_on_monomials(dim, q):
    pts, wts = quadrature.simplex_rule(dim, q)
    assert len(wts) == quadrature.points_per_direction(q) ** dim
    assert np.all(wts > 0)
    assert np.all(pts > 0) and np.all(pts.sum(axis=1) < 1)
    assert abs(wts.sum() - 1.0 / factorial(dim)) < 1e-15
    for total in range(q + 1):
        for alpha in itertools.product(range(total + 1), repeat=dim):
            if sum(alpha) != total:
                continue
            val = np.sum(wts * np.prod(pts ** np.asarray(alpha), axis=1))
            assert abs(val - monomial_integral(alpha)) < 1e-15, (alpha, val)


def test_simplex_rule_not_exact_beyond_degree():
    # a deliberately too-low rule misses a high monomial: the exactness test has teeth
    pts, wts = quadrature.simplex_rule(2, 2)
    alpha = (4, 0)
    val = np.sum(wts * np.prod(pts ** np.asarray(alpha), axis=1))
    assert abs(val - monomial_integral(alpha)) > 1e-6


def _lattice(dim, p):
    return np.asarray(basis.multi_indices(dim, p), dtype=float) / p


@pytest.mark.parametrize("dim,p", [(1, 3), (2, 1), (2, 2), (2, 4), (2, 6), (3, 1), (3, 2), (3, 4)])
def test_basis_nodal_and_partition_of_unity(dim, p):
    nodes = _lattice(dim, p)
    n = len(nodes)
    assert n == comb(p + dim, dim)
    V = np.array([basis.basis_at(dim, p, x)[0] for x in nodes])
    np.testing.assert_allclose(V, np.eye(n), atol=1e-12)
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.dirichlet(np.ones(dim + 1))[1:]
        v, g = basis.basis_at(dim, p, x)
        assert abs(v.sum() - 1.0) < 1e-12
        np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-10)


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (2, 6), (3, 2), (3, 4)])
def test_basis_gradient_matches_central_differences(dim, p):
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(3):
        x = rng.dirichlet(np.ones(dim + 1) * 2)[1:]
        _, g = basis.basis_at(dim, p, x)
        for k in range(dim):
            e = np.zeros(dim)
            e[k] = h
            fd = (basis.basis_at(dim, p, x + e)[0] - basis.basis_at(dim, p, x - e)[0]) / (2 * h)
            np.testing.assert_allclose(g[k], fd, atol=1e-6 * max(1, np.abs(g).max()))


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2)])
def test_basis_reproduces_polynomials(dim, p):
    """Interpolating any monomial of degree <= p at the nodes reproduces it exactly."""
    nodes = _lattice(dim, p)
    rng = np.random.default_rng(7)
    for alpha in itertools.product(range(p + 1), repeat=dim):
        if sum(alpha) > p:
            continue
        coeff = np.prod(nodes ** np.asarray(alpha), axis=1)
        x = rng.dirichlet(np.ones(dim + 1))[1:]
        v, g = basis.basis_at(dim, p, x)
        exact = np.prod(x ** np.asarray(alpha))
        assert abs(v @ coeff - exact) < 1e-12
        for k in range(dim):
            a = list(alpha)
            if a[k] == 0:
                dexact = 0.0
            else:
                a[k] -= 1
                dexact = alpha[k] * np.prod(x ** np.asarray(a))
            assert abs(g[k] @ coeff - dexact) < 1e-10


def test_table_sizes_match_paper():
    """Local DoF counts and derivative-term counts of Table "action_param_space"."""
    with open(os.path.join(GOLDEN, "action_param_space.json")) as f:
        rows = json.load(f)["rows"]
    for row in rows:
        n = len(basis.multi_indices(row["d"], row["degree"]))
        assert n == row["n_local"], row
        nc = row["d"] if row["vector"] else 1
        # value-only forms use one derivative term per component; gradient forms d per
        # component and per trial field
        terms = row["trial_fields"] * nc * (1 if row["kind"] == "mass" else row["d"])
        if row["kind"] == "helmholtz":
            terms = 1 + row["d"]
        assert terms == row["n_deriv"], row


# ---------------------------------------------------------------- symmetric rules
SYM = [(2, 2, 3), (2, 4, 6), (2, 6, 12), (2, 8, 16), (3, 2, 4), (3, 5, 14), (3, 6, 24)]


@pytest.mark.parametrize("dim,q,npts", SYM)
def test_symmetric_rules_exact_positive_invariant(dim, q, npts):
    from oracle.symmetric import symmetric_rule
    pts, wts = symmetric_rule(dim, q)
    assert len(wts) == npts
    assert np.all(wts > 0) and np.all(pts > 0) and np.all(pts.sum(axis=1) < 1)
    assert abs(wts.sum() - 1.0 / factorial(dim)) < 1e-15
    for total in range(q + 1):
        for alpha in itertools.product(range(total + 1), repeat=dim):
            if sum(alpha) != total:
                continue
            val = np.sum(wts * np.prod(pts ** np.asarray(alpha), axis=1))
            assert abs(val - monomial_integral(alpha)) < 1e-15, (alpha, val)
    # invariance: permuting the barycentric coordinates maps the rule onto itself
    lam = np.concatenate([1 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    key = {tuple(np.round(l, 13)): w for l, w in zip(lam, wts)}
    for perm in itertools.permutations(range(dim + 1)):
        for l, w in zip(lam[:, perm], wts):
            assert abs(key[tuple(np.round(l, 13))] - w) < 1e-16


def test_symmetric_rule_sizes_match_paper_point_counts():
    """Table "action_param_space": Mass P3 and P4 on triangles use Q = 12 and 16 points,
    the sizes of the degree-6 and degree-8 fully symmetric rules (2p for mass)."""
    from oracle.symmetric import symmetric_rule
    with open(os.path.join(GOLDEN, "action_param_space.json")) as f:
        rows = {(r["d"], r["kind"], r["degree"]): r for r in json.load(f)["rows"]}
    for p in (3, 4):
        assert len(symmetric_rule(2, 2 * p)[1]) == rows[(2, "mass", p)]["Q_paper"]


def test_symmetric_family_falls_back_to_conical():
    from oracle.symmetric import symmetric_rule
    pts, wts = symmetric_rule(3, 7)
    p2, w2 = quadrature.simplex_rule(3, 7)
    assert np.array_equal(pts, p2) and np.array_equal(wts, w2)
