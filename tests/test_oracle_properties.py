"""Property tests of the oracle's invariants over random small meshes (hypothesis):
dimension, degree, mesh size, jitter seed and field draws vary; each property is
one the definitions fix for every such mesh (no GPU)."""

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from feinputs import lame_fields, shuffled_mesh, structured_mesh, uniform_field  # noqa: E402
from feinputs.fields import node_positions  # noqa: E402
from oracle import Oracle  # noqa: E402

meshes = st.tuples(st.sampled_from([2, 3]), st.integers(1, 3), st.integers(1, 3), st.integers(0, 10_000))
SETTINGS = settings(max_examples=25, deadline=None)


def make(dim, N, p, seed):
    return structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)


def vec_field(pos, f):
    return np.ascontiguousarray(f(pos)).reshape(-1)


@SETTINGS
@given(meshes)
def test_mass_of_one_is_the_volume(oracle_built, case):
    """sum(M 1) = |Omega| = 1 for any jitter and degree (degree-2p rule: exact)."""
    dim, N, p, seed = case
    m = make(dim, N, p, seed)
    y = Oracle.from_mesh(m, 2 * p).mass(np.ones(m.n_nodes))
    assert abs(y.sum() - 1.0) < 1e-12


@SETTINGS
@given(meshes, st.integers(0, 2**31 - 1))
def test_mass_and_elasticity_are_symmetric(oracle_built, case, draw):
    """v . A u = u . A v for random u, v (both forms are symmetric bilinear forms)."""
    dim, N, p, seed = case
    m = make(dim, N, p, seed)
    o = Oracle.from_mesh(m, 2 * p)
    rng = np.random.default_rng(draw)
    u, v = rng.uniform(-1, 1, m.n_nodes), rng.uniform(-1, 1, m.n_nodes)
    assert abs(v @ o.mass(u) - u @ o.mass(v)) <= 1e-13 * (abs(v @ o.mass(u)) + 1e-30) + 1e-15
    U, V = rng.uniform(-1, 1, m.n_nodes * dim), rng.uniform(-1, 1, m.n_nodes * dim)
    a, b = V @ o.elasticity(U, 1.25, 1.0), U @ o.elasticity(V, 1.25, 1.0)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


@SETTINGS
@given(meshes, st.integers(0, 2**31 - 1))
def test_elasticity_annihilates_rigid_motions(oracle_built, case, draw):
    """u = a + B x with B skew: zero strain, so A u = 0 to rounding."""
    dim, N, p, seed = case
    m = make(dim, N, p, seed)
    o = Oracle.from_mesh(m, max(2 * (p - 1), 0))
    rng = np.random.default_rng(draw)
    a = rng.normal(size=dim)
    B = rng.normal(size=(dim, dim))
    B = B - B.T
    u = vec_field(node_positions(m), lambda x: a[None, :] + x @ B.T)
    scale = np.abs(o.elasticity(uniform_field(m.n_nodes * dim, 1), 1.25, 1.0)).max()
    assert np.abs(o.elasticity(u, 1.25, 1.0)).max() < 1e-12 * scale * (1 + np.abs(u).max())


@SETTINGS
@given(meshes, st.integers(0, 2**31 - 1))
def test_hyperelastic_residuals_vanish_at_rest_and_under_rotation(oracle_built, case, draw):
    """Neo-Hookean and St. Venant-Kirchhoff: r(0) = 0, and r = 0 for a finite
    rotation u = (R - I) x (F = R is stress free for both laws)."""
    dim, N, p, seed = case
    m = make(dim, N, p, seed)
    o = Oracle.from_mesh(m, 2 * p)
    mu, lam = lame_fields(m.n_cells, draw % 1000)
    zero = np.zeros(m.n_nodes * dim)
    assert np.abs(o.nh_residual(zero, mu, lam)).max() == 0.0
    assert np.abs(o.svk_residual(zero, mu, lam)).max() == 0.0
    rng = np.random.default_rng(draw)
    if dim == 2:
        t = rng.uniform(-np.pi, np.pi)
        R = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    else:
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        R = Q * np.sign(np.linalg.det(Q))
    u = vec_field(node_positions(m), lambda x: x @ (R - np.eye(dim)).T)
    # stiffness scale: the linear action with the largest Lame parameters drawn (<= 10, 2)
    scale = np.abs(o.elasticity(uniform_field(m.n_nodes * dim, 3), 10.0, 2.0)).max()
    assert np.abs(o.nh_residual(u, mu, lam)).max() < 1e-11 * max(scale, 1.0)
    assert np.abs(o.svk_residual(u, mu, lam)).max() < 1e-11 * max(scale, 1.0)


@SETTINGS
@given(meshes, st.integers(0, 2**31 - 1))
def test_actions_are_numbering_invariant(oracle_built, case, draw):
    """Renumbering cells, vertices and nodes at random renumbers the action and
    changes nothing else (the action is a sum over cells of local terms)."""
    dim, N, p, seed = case
    m = make(dim, N, p, seed)
    s = shuffled_mesh(m, draw % 100_000)
    node_old = s.meta["node_old"]
    q = max(2 * (p - 1), 0)
    u = uniform_field(m.n_nodes * dim, draw % 1000)
    y = Oracle.from_mesh(m, q).elasticity(u, 1.25, 1.0)
    us = u.reshape(-1, dim)[node_old].reshape(-1)        # node k of s is node node_old[k] of m
    ys = Oracle.from_mesh(s, q).elasticity(us, 1.25, 1.0)
    assert np.abs(ys.reshape(-1, dim) - y.reshape(-1, dim)[node_old]).max() <= 1e-13 * np.abs(y).max()
