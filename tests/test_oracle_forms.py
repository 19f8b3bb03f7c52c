"""Pins for the oracle's actions (no GPU): closed forms, invariants, exact rational
assembly on tiny meshes and finite differences.

Forms: Appendix A (Mass, Elasticity) and the compressible Neo-Hookean law that
replaces the appendix's St. Venant-Kirchhoff hyperelasticity; the action is
Algorithm 2.  Each pin is chosen so that a dropped term, a wrong sign/index or a
transposed operand in the oracle fails it.
"""

from fractions import Fraction

import numpy as np
import pytest

from feinputs import structured_mesh, uniform_field, lame_fields
from feinputs.fields import node_positions, sinusoid_displacement
from oracle import Oracle

from exact_fe import assemble, element_mass


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------- mass
@pytest.mark.parametrize("dim,p,q", [(2, 2, 4), (2, 3, 6), (3, 2, 4), (2, 4, 8)])
def test_mass_closed_forms(oracle_built, dim, p, q):
    """1.M1 = |Omega| = 1; 1.Mx = int x = 1/2; x.Mx = 1/3; (xy).M(xy) = 1/9 (P2+ and
    a degree-4+ rule reproduce them exactly on any jittered mesh)."""
    m = structured_mesh(dim, 5, p, jitter=0.2 if dim == 2 else 0.15, seed=11)
    o = Oracle.from_mesh(m, q)
    pos = node_positions(m)
    one = np.ones(m.n_nodes)
    x, y = pos[:, 0], pos[:, 1]
    assert abs(o.mass(one).sum() - 1.0) < 1e-13
    assert abs(one @ o.mass(x) - 0.5) < 1e-13
    assert abs(x @ o.mass(x) - 1.0 / 3.0) < 1e-13
    assert abs((x * y) @ o.mass(x * y) - 1.0 / 9.0) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_p1_element_textbook(oracle_built, dim):
    """P1 element mass matrix |T| (1 + delta_ij) / ((d+1)(d+2)) on a single cell."""
    X = np.array([[0.1, 0.0, 0.2], [1.3, 0.2, 0.1], [0.3, 1.1, 0.0], [0.2, 0.3, 0.9]])[: dim + 1, :dim]
    c2v = np.arange(dim + 1, dtype=np.int32)[None, :]
    # P1 local node order (alpha_1 outer .. alpha_d inner): map local nodes to vertices
    from feinputs.mesh import local_multi_indices
    al = local_multi_indices(dim, 1)
    c2n = np.array([[0 if a.sum() == 0 else 1 + int(np.argmax(a)) for a in al]], dtype=np.int32)
    o = Oracle(dim, 1, 2, X, c2v, c2n, dim + 1)
    M = o.dense(o.mass, dim + 1)
    vol = abs(np.linalg.det((X[1:] - X[0]).T)) / (2 if dim == 2 else 6)
    ref = vol * (np.ones((dim + 1, dim + 1)) + np.eye(dim + 1)) / ((dim + 1) * (dim + 2))
    np.testing.assert_allclose(M, ref, rtol=1e-13, atol=1e-16)


def _rational_mesh(dim, N, p, seed):
    """Structured mesh whose interior vertices carry rational jitter (exact inputs)."""
    m = structured_mesh(dim, N, p, jitter=0.0)
    rng = np.random.default_rng(seed)
    Xq = [[Fraction(int(round(c * N)), N) for c in v] for v in m.coords]
    for v in range(len(Xq)):
        interior = all(0 < Fraction(c) < 1 for c in Xq[v])
        if interior:
            Xq[v] = [c + Fraction(int(rng.integers(-3, 4)), 20 * N) for c in Xq[v]]
    coords = np.array([[float(c) for c in v] for v in Xq])
    m.coords = coords
    cells = [[Xq[v] for v in cell] for cell in m.cell2vertex]
    return m, cells


def test_mass_dense_matches_exact_rational(oracle_built):
    m, cells = _rational_mesh(2, 2, 2, seed=1)
    o = Oracle.from_mesh(m, 4)
    A = o.dense(o.mass, m.n_nodes)
    E = assemble(cells, m.cell2node, m.n_nodes, 2, "mass")
    Ef = np.array([[float(v) for v in row] for row in E])
    assert rel(A, Ef) < 1e-13


def test_mass_element_p3_exact(oracle_built):
    X = [[Fraction(0), Fraction(0)], [Fraction(5, 4), Fraction(1, 7)], [Fraction(2, 9), Fraction(1)]]
    c2v = np.array([[0, 1, 2]], dtype=np.int32)
    c2n = np.arange(10, dtype=np.int32)[None, :]
    o = Oracle(2, 3, 6, np.array([[float(c) for c in v] for v in X]), c2v, c2n, 10)
    M = o.dense(o.mass, 10)
    E = np.array([[float(v) for v in row] for row in element_mass(X, 3)])
    assert rel(M, E) < 1e-13


# ---------------------------------------------------------------- elasticity
def _vec_field(pos, fn):
    return np.ascontiguousarray(fn(pos).reshape(-1))


@pytest.mark.parametrize("dim,p,q", [(2, 2, 2), (3, 2, 2), (3, 1, 2), (2, 4, 6)])
def test_elasticity_rigid_modes(oracle_built, dim, p, q):
    m = structured_mesh(dim, 3, p, jitter=0.15, seed=4)
    o = Oracle.from_mesh(m, q)
    pos = node_positions(m)
    rng = np.random.default_rng(0)
    a = rng.normal(size=dim)
    B = rng.normal(size=(dim, dim))
    B = B - B.T
    u = _vec_field(pos, lambda x: a[None, :] + x @ B.T)
    y = o.elasticity(u, 1.25, 1.0)
    scale = np.abs(o.elasticity(uniform_field(len(u), 1), 1.25, 1.0)).max()
    assert np.abs(y).max() < 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_elasticity_patch_and_energy(oracle_built, dim):
    """Affine u: interior rows vanish (patch test); u=(x,0,..): u.Au = (lambda+2mu)|Omega|."""
    m = structured_mesh(dim, 3, 2, jitter=0.15, seed=8)
    o = Oracle.from_mesh(m, 2)
    pos = node_positions(m)
    rng = np.random.default_rng(2)
    G = rng.normal(size=(dim, dim))
    c = rng.normal(size=dim)
    u = _vec_field(pos, lambda x: c[None, :] + x @ G.T)
    y = o.elasticity(u, 1.25, 1.0).reshape(-1, dim)
    interior = ~m.boundary_nodes()
    assert np.abs(y[interior]).max() < 1e-12 * np.abs(y).max()
    u1 = _vec_field(pos, lambda x: np.stack([x[:, 0]] + [0 * x[:, 0]] * (dim - 1), axis=1))
    assert abs(u1 @ o.elasticity(u1, 1.25, 1.0) - 3.25) < 1e-12
    # the paper's constants lambda = 0, mu = 1/2 give sigma = eps and energy 1
    assert abs(u1 @ o.elasticity(u1, 0.0, 0.5) - 1.0) < 1e-12
    # shear u = (y, 0): eps_xy = 1/2, sigma:eps = 2 mu eps:eps = mu
    us = _vec_field(pos, lambda x: np.stack([x[:, 1]] + [0 * x[:, 0]] * (dim - 1), axis=1))
    assert abs(us @ o.elasticity(us, 1.25, 1.0) - 1.0) < 1e-12


def test_elasticity_symmetry(oracle_built):
    m = structured_mesh(3, 2, 2, jitter=0.15, seed=5)
    o = Oracle.from_mesh(m, 2)
    n = m.n_nodes * 3
    u, v = uniform_field(n, 1), uniform_field(n, 2)
    a, b = v @ o.elasticity(u, 1.25, 1.0), u @ o.elasticity(v, 1.25, 1.0)
    assert abs(a - b) < 1e-13 * abs(a)


@pytest.mark.parametrize("dim,N,p", [(2, 2, 2), (3, 1, 2), (3, 1, 1)])
def test_elasticity_dense_matches_exact_rational(oracle_built, dim, N, p):
    m, cells = _rational_mesh(dim, N, p, seed=3)
    if dim == 3 and N == 1:
        # no interior vertex at N=1: perturb the corners rationally instead
        rng = np.random.default_rng(9)
        from exact_fe import ExactCell  # noqa: F401
        Xq = [[Fraction(int(round(c)), 1) + Fraction(int(rng.integers(-2, 3)), 40) for c in v]
              for v in m.coords]
        m.coords = np.array([[float(c) for c in v] for v in Xq])
        cells = [[Xq[v] for v in cell] for cell in m.cell2vertex]
    o = Oracle.from_mesh(m, 2 * (p - 1))
    n = m.n_nodes * dim
    A = o.dense(lambda u: o.elasticity(u, Fraction(5, 4), 1.0), n)
    E = assemble(cells, m.cell2node, m.n_nodes, p, "elasticity", ncomp=dim,
                 lam=Fraction(5, 4), mu=1)
    Ef = np.array([[float(v) for v in row] for row in E])
    assert rel(A, Ef) < 1e-12


# ---------------------------------------------------------------- Neo-Hookean
def _nh_setup(dim=2, N=3, p=3, q=6, seed=21):
    m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)
    o = Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, seed + 1)
    return m, o, mu, lam


@pytest.mark.parametrize("dim", [2, 3])
def test_nh_residual_zero_at_rest_and_under_rotation(oracle_built, dim):
    m, o, mu, lam = _nh_setup(dim=dim, N=2, p=2, q=4)
    n = m.n_nodes * dim
    assert np.abs(o.nh_residual(np.zeros(n), mu, lam)).max() == 0.0
    th = 0.7
    if dim == 2:
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    else:
        R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
        R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    pos = node_positions(m)
    u = _vec_field(pos, lambda x: x @ (R - np.eye(dim)).T)
    r = o.nh_residual(u, mu, lam)
    ref = np.abs(o.nh_residual(0.01 * uniform_field(n, 3), mu, lam)).max()
    assert np.abs(r).max() < 1e-12 * ref


def test_nh_homogeneous_deformation_interior_rows_vanish(oracle_built):
    m, o, mu, lam = _nh_setup(N=4, p=2, q=4)
    mu[:] = 1.3
    lam[:] = 4.0   # homogeneous material: div P = 0 for constant F
    pos = node_positions(m)
    G = np.array([[0.1, 0.05], [-0.02, 0.15]])
    u = _vec_field(pos, lambda x: x @ G.T)
    r = o.nh_residual(u, mu, lam).reshape(-1, 2)
    interior = ~m.boundary_nodes()
    assert np.abs(r[interior]).max() < 1e-13 * np.abs(r).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_nh_homogeneous_stretch_energy_and_traction_closed_form(oracle_built, dim):
    """Absolute pins of the Neo-Hookean law.  Under the homogeneous stretch
    u_k = a_k x_k the deformation gradient is F = diag(1 + a_k) everywhere, so
    (1) the energy is Pi = Psi(F) |Omega| with |Omega| = 1, Psi = mu/2 (tr F^T F - d)
    - mu ln J + lambda/2 (ln J)^2, J = det F; and (2) with P constant, the x-rows of
    the residual summed over the nodes of the face x = 1 equal int_Omega P_1k
    d_k psi = P_11 (psi = the sum of those nodes' basis functions: 1 on x = 1, 0 on
    x = 0, and its traces on the faces normal to the other axes cancel in
    pairs because the boundary vertices are not jittered), with
    P_11 = mu (F_11 - 1/F_11) + lambda ln J / F_11.  A volumetric term misread
    consistently in the energy and the residual (J - 1 for ln J, say) passes the
    energy-gradient check but fails both closed forms."""
    m = structured_mesh(dim, 3, 2, jitter=0.2 if dim == 2 else 0.15, seed=61)
    o = Oracle.from_mesh(m, 4)
    mu_v, lam_v = 0.7, 3.1
    mu = np.full(m.n_cells, mu_v)
    lam = np.full(m.n_cells, lam_v)
    a = np.array([0.13, -0.08, 0.21])[:dim]
    pos = node_positions(m)
    u = _vec_field(pos, lambda x: x * a[None, :])
    f = 1.0 + a
    J = float(np.prod(f))
    psi = mu_v / 2 * (np.sum(f ** 2) - dim) - mu_v * np.log(J) + lam_v / 2 * np.log(J) ** 2
    assert abs(o.nh_energy(u, mu, lam).sum() - psi) < 1e-14 * max(1.0, abs(psi))
    r = o.nh_residual(u, mu, lam).reshape(-1, dim)
    face = np.abs(pos[:, 0] - 1.0) < 1e-12
    p11 = mu_v * (f[0] - 1.0 / f[0]) + lam_v * np.log(J) / f[0]
    assert abs(r[face, 0].sum() - p11) < 1e-13 * abs(p11)
    # and the other components: P is diagonal, so the face sums of the y (and z)
    # rows vanish
    for k in range(1, dim):
        assert abs(r[face, k].sum()) < 1e-13 * abs(p11)


def test_nh_residual_is_energy_gradient(oracle_built):
    m, o, mu, lam = _nh_setup()
    n = m.n_nodes * 2
    u = sinusoid_displacement(m, 31)
    d = uniform_field(n, 32)
    h = 1e-6
    fd = (o.nh_energy(u + h * d, mu, lam).sum() - o.nh_energy(u - h * d, mu, lam).sum()) / (2 * h)
    an = o.nh_residual(u, mu, lam) @ d
    assert abs(fd - an) < 1e-7 * abs(an)


def test_nh_jacobian_is_residual_derivative(oracle_built):
    """Central-difference check of the Jacobian action: J(u) du = (r(u + h du) - r(u - h du)) / 2h, h = 1e-6."""
    m, o, mu, lam = _nh_setup()
    n = m.n_nodes * 2
    u = sinusoid_displacement(m, 41)
    du = uniform_field(n, 42)
    h = 1e-6
    fd = (o.nh_residual(u + h * du, mu, lam) - o.nh_residual(u - h * du, mu, lam)) / (2 * h)
    an = o.nh_jacobian(u, du, mu, lam)
    assert rel(an, fd) < 1e-7


def test_nh_jacobian_symmetric_and_linearises_to_elasticity(oracle_built):
    m, o, mu, lam = _nh_setup()
    n = m.n_nodes * 2
    u = sinusoid_displacement(m, 51)
    v, w = uniform_field(n, 52), uniform_field(n, 53)
    a, b = w @ o.nh_jacobian(u, v, mu, lam), v @ o.nh_jacobian(u, w, mu, lam)
    assert abs(a - b) < 1e-12 * abs(a)
    mu_c = np.full(m.n_cells, 1.0)
    lam_c = np.full(m.n_cells, 1.25)
    j0 = o.nh_jacobian(np.zeros(n), v, mu_c, lam_c)
    el = o.elasticity(v, 1.25, 1.0)
    assert rel(j0, el) < 1e-13


def test_nh_adjoint_pins(oracle_built):
    """J^T w equals J w (hyperelastic tangent is symmetric, computed here by two
    different routes); r is linear in (mu, lambda) so w.r = sum mu dmu + lam dlam
    exactly; central differences in one cell's mu/lambda are exact up to roundoff."""
    m, o, mu, lam = _nh_setup(N=2, p=3, q=6)
    n = m.n_nodes * 2
    u = sinusoid_displacement(m, 61)
    w = uniform_field(n, 62)
    jtw, dmu, dlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, o.nh_jacobian(u, w, mu, lam)) < 1e-12
    wr = w @ o.nh_residual(u, mu, lam)
    assert abs(wr - (mu @ dmu + lam @ dlam)) < 1e-12 * max(abs(wr), np.abs(mu * dmu).sum())
    h = 1e-3
    for c in (0, 3, m.n_cells - 1):
        e = np.zeros(m.n_cells)
        e[c] = h
        fmu = (w @ o.nh_residual(u, mu + e, lam) - w @ o.nh_residual(u, mu - e, lam)) / (2 * h)
        flam = (w @ o.nh_residual(u, mu, lam + e) - w @ o.nh_residual(u, mu, lam - e)) / (2 * h)
        assert abs(fmu - dmu[c]) < 1e-9 * max(1.0, abs(dmu[c]))
        assert abs(flam - dlam[c]) < 1e-9 * max(1.0, abs(dlam[c]))


def test_oracle_threads_agree(oracle_built):
    m, o, mu, lam = _nh_setup(N=6, p=4, q=8)
    u = sinusoid_displacement(m, 71)
    a = o.nh_residual(u, mu, lam, threads=1)
    b = o.nh_residual(u, mu, lam, threads=4)
    assert rel(b, a) < 1e-14


def test_oracle_flags_degenerate_cell(oracle_built):
    m = structured_mesh(2, 2, 1)
    m.coords[m.cell2vertex[0, 1]] = m.coords[m.cell2vertex[0, 0]]  # collapse an edge
    o = Oracle.from_mesh(m, 2)
    from oracle import OracleError
    with pytest.raises(OracleError):
        o.mass(np.ones(m.n_nodes))
