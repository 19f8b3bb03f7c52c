"""Pins for the oracle's Laplacian, Helmholtz and St. Venant-Kirchhoff forms (no GPU).

Forms of Appendix A: Laplacian a = int grad u . grad v, Helmholtz
a = int (grad u . grad v + u v), and the St. Venant-Kirchhoff hyperelastic law
Psi = lambda/2 (tr E)^2 + mu tr(E^2), S = dPsi/dE, P = F S, with the residual
r = int P : grad v and its linearisation.  Pins: closed-form integrals, the
kernel of the operator (constants, rigid motions), the patch test, the P1
cotangent formula, exact rational assembly, the energy gradient and the
Jacobian by central differences, symmetry, and the linearisation at u = 0.
"""

from fractions import Fraction
import math

import numpy as np
import pytest

from feinputs import structured_mesh, uniform_field, lame_fields
from feinputs.fields import node_positions, sinusoid_displacement
from oracle import Oracle

from exact_fe import assemble


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _vec_field(pos, fn):
    return np.ascontiguousarray(fn(pos).reshape(-1))


# ---------------------------------------------------------------- Laplacian
@pytest.mark.parametrize("dim,p,q", [(2, 1, 0), (2, 2, 2), (2, 4, 6), (3, 2, 2), (3, 3, 4)])
def test_laplace_kernel_and_closed_forms(oracle_built, dim, p, q):
    """L 1 = 0; x.Lx = int |grad x|^2 = 1; for P >= 2: x^2.L x^2 = int 4 x^2 = 4/3 and
    (xy).L(xy) = int (x^2 + y^2) = 2/3 (exact: P_p reproduces them and the rule is
    exact to degree 2(p-1))."""
    m = structured_mesh(dim, 4, p, jitter=0.2 if dim == 2 else 0.15, seed=13)
    o = Oracle.from_mesh(m, q)
    pos = node_positions(m)
    x, y = pos[:, 0], pos[:, 1]
    scale = np.abs(o.laplace(uniform_field(m.n_nodes, 1))).max()
    assert np.abs(o.laplace(np.ones(m.n_nodes))).max() < 1e-13 * scale
    assert abs(x @ o.laplace(x) - 1.0) < 1e-12
    if p >= 2:
        assert abs((x * x) @ o.laplace(x * x) - 4.0 / 3.0) < 1e-12
        assert abs((x * y) @ o.laplace(x * y) - 2.0 / 3.0) < 1e-12


def test_laplace_patch_and_symmetry(oracle_built):
    m = structured_mesh(3, 3, 2, jitter=0.15, seed=14)
    o = Oracle.from_mesh(m, 2)
    pos = node_positions(m)
    u = 0.3 + pos @ np.array([1.0, -2.0, 0.5])
    r = o.laplace(u)
    assert np.abs(r[~m.boundary_nodes()]).max() < 1e-12 * np.abs(r).max()
    a, b = uniform_field(m.n_nodes, 2), uniform_field(m.n_nodes, 3)
    assert abs(b @ o.laplace(a) - a @ o.laplace(b)) < 1e-13 * abs(b @ o.laplace(a))


def test_laplace_p1_cotangent_formula(oracle_built):
    """P1 triangle: K_ij = -cot(theta_k)/2 (theta_k the angle opposite edge ij),
    K_ii = -sum_j K_ij — the textbook closed form."""
    X = np.array([[0.1, 0.0], [1.3, 0.2], [0.4, 0.9]])
    o = Oracle(2, 1, 0, X, np.array([[0, 1, 2]], dtype=np.int32), np.array([[0, 1, 2]], dtype=np.int32), 3)
    K = o.dense(o.laplace, 3)
    ref = np.zeros((3, 3))
    for k in range(3):
        i, j = [v for v in range(3) if v != k]
        a, b = X[i] - X[k], X[j] - X[k]
        cot = (a @ b) / abs(a[0] * b[1] - a[1] * b[0])
        ref[i, j] = ref[j, i] = -0.5 * cot
    for i in range(3):
        ref[i, i] = -ref[i].sum()
    # local P1 nodes follow the multi-index order (alpha_1 outer): vertices 0, 2, 1
    perm = [0, 2, 1]
    np.testing.assert_allclose(K, ref[np.ix_(perm, perm)], rtol=1e-13, atol=1e-15)


def _rational_mesh(dim, N, p, seed):
    m = structured_mesh(dim, N, p, jitter=0.0)
    rng = np.random.default_rng(seed)
    Xq = [[Fraction(int(round(c * N)), N) for c in v] for v in m.coords]
    for v in range(len(Xq)):
        Xq[v] = [c + Fraction(int(rng.integers(-2, 3)), 40 * N) for c in Xq[v]]
    m.coords = np.array([[float(c) for c in v] for v in Xq])
    return m, [[Xq[v] for v in cell] for cell in m.cell2vertex]


@pytest.mark.parametrize("kind,dim,N,p", [("laplace", 2, 2, 2), ("laplace", 3, 1, 2),
                                          ("helmholtz", 2, 2, 2), ("helmholtz", 3, 1, 1)])
def test_laplace_helmholtz_dense_match_exact_rational(oracle_built, kind, dim, N, p):
    m, cells = _rational_mesh(dim, N, p, seed=5)
    o = Oracle.from_mesh(m, 2 * p)
    A = o.dense(getattr(o, kind), m.n_nodes)
    E = assemble(cells, m.cell2node, m.n_nodes, p, kind)
    Ef = np.array([[float(v) for v in row] for row in E])
    assert rel(A, Ef) < 1e-12


# ---------------------------------------------------------------- Helmholtz
@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2)])
def test_helmholtz_closed_forms(oracle_built, dim, p):
    """sum H 1 = |Omega| = 1 (the gradient term vanishes); x.Hx = 1 + 1/3."""
    m = structured_mesh(dim, 4, p, jitter=0.2 if dim == 2 else 0.15, seed=15)
    o = Oracle.from_mesh(m, 2 * p)
    x = node_positions(m)[:, 0]
    assert abs(o.helmholtz(np.ones(m.n_nodes)).sum() - 1.0) < 1e-13
    assert abs(x @ o.helmholtz(x) - 4.0 / 3.0) < 1e-12


# ---------------------------------------------------------------- St. Venant-Kirchhoff
def _svk_setup(dim=2, N=3, p=3, q=6, seed=23):
    m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)
    o = Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, seed + 1)
    return m, o, mu, lam


@pytest.mark.parametrize("dim", [2, 3])
def test_svk_residual_zero_at_rest_and_under_rotation(oracle_built, dim):
    """E = 0 for u = 0 and for a finite rigid rotation F = R, so S = 0 and r = 0."""
    m, o, mu, lam = _svk_setup(dim=dim, N=2, p=2, q=2)
    n = m.n_nodes * dim
    assert np.abs(o.svk_residual(np.zeros(n), mu, lam)).max() == 0.0
    th = 0.9
    if dim == 2:
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    else:
        R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
        R = R @ np.array([[1, 0, 0], [0, np.cos(0.5), -np.sin(0.5)], [0, np.sin(0.5), np.cos(0.5)]])
    u = _vec_field(node_positions(m), lambda x: x @ (R - np.eye(dim)).T)
    ref = np.abs(o.svk_residual(0.05 * uniform_field(n, 3), mu, lam)).max()
    assert np.abs(o.svk_residual(u, mu, lam)).max() < 1e-12 * ref


def test_svk_homogeneous_stretch_energy_and_patch(oracle_built):
    """u = (a x, 0): F = diag(1+a, 1), E = diag(e, 0) with e = ((1+a)^2 - 1)/2, so
    Pi = (lambda/2 + mu) e^2 |Omega|; constant F with constant material gives
    vanishing interior rows."""
    m, o, mu, lam = _svk_setup(N=4, p=2, q=4)
    mu[:] = 0.7
    lam[:] = 2.5
    a = 0.3
    pos = node_positions(m)
    u = _vec_field(pos, lambda x: np.stack([a * x[:, 0], 0 * x[:, 0]], axis=1))
    e = ((1 + a) ** 2 - 1) / 2
    assert abs(o.svk_energy(u, mu, lam).sum() - (0.5 * 2.5 + 0.7) * e * e) < 1e-13
    G = np.array([[0.12, -0.07], [0.04, 0.2]])
    r = o.svk_residual(_vec_field(pos, lambda x: x @ G.T), mu, lam).reshape(-1, 2)
    assert np.abs(r[~m.boundary_nodes()]).max() < 1e-13 * np.abs(r).max()


def _d5(f, h):
    """Five-point central difference f'(0): exact for polynomials of degree <= 4."""
    return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)


def test_svk_residual_is_energy_gradient(oracle_built):
    """Pi(u + t d) is a quartic in t (E is quadratic in grad u, Psi quadratic in E,
    the quadrature a finite sum), so the five-point stencil gives r(u).d up to
    roundoff for any step."""
    m, o, mu, lam = _svk_setup()
    n = m.n_nodes * 2
    u = sinusoid_displacement(m, 71)
    d = uniform_field(n, 72)
    fd = _d5(lambda t: o.svk_energy(u + t * d, mu, lam).sum(), 1e-2)
    an = o.svk_residual(u, mu, lam) @ d
    scale = np.abs(o.svk_residual(u, mu, lam)) @ np.abs(d)
    assert abs(fd - an) < 1e-11 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_svk_jacobian_is_residual_derivative_and_symmetric(oracle_built, dim):
    m, o, mu, lam = _svk_setup(dim=dim, N=2, p=2, q=4)
    n = m.n_nodes * dim
    u = sinusoid_displacement(m, 81)
    du, w = uniform_field(n, 82), uniform_field(n, 83)
    # r(u + t du) is a cubic in t: the five-point stencil is exact up to roundoff
    fd = _d5(lambda t: o.svk_residual(u + t * du, mu, lam), 1e-2)
    an = o.svk_jacobian(u, du, mu, lam)
    assert rel(an, fd) < 1e-10
    # and the plain central difference with h = 1e-6, whose truncation and roundoff stay below 1e-7
    h = 1e-6
    fd2 = (o.svk_residual(u + h * du, mu, lam) - o.svk_residual(u - h * du, mu, lam)) / (2 * h)
    assert rel(an, fd2) < 1e-7
    a, b = w @ o.svk_jacobian(u, du, mu, lam), du @ o.svk_jacobian(u, w, mu, lam)
    assert abs(a - b) < 1e-12 * abs(a)


def test_svk_jacobian_at_rest_is_linear_elasticity(oracle_built):
    """At u = 0: F = I, S = 0, dE = sym(H), dP = dS = sigma(du)."""
    m, o, mu, lam = _svk_setup(dim=3, N=2, p=2, q=2)
    n = m.n_nodes * 3
    v = uniform_field(n, 91)
    j0 = o.svk_jacobian(np.zeros(n), v, np.full(m.n_cells, 1.0), np.full(m.n_cells, 1.25))
    assert rel(j0, o.elasticity(v, 1.25, 1.0)) < 1e-13
