"""Locality orderings (fe_order_cells_morton, fe_order_first_touch) on the CPU:
against plain Python restatements of their definitions, as permutations, by the
locality they restore on a randomly numbered mesh, and by operator invariance
(the oracle's action on the renumbered mesh is the renumbered action)."""

import numpy as np
import pytest

import oracle
from feinputs import structured_mesh, shuffled_mesh, uniform_field


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build()
    oracle.build()
    import paper_2506_17471_gb300 as fe
    return fe


def _morton_key(q, dim, bits):
    """Bit interleaving written out bit by bit: bit b of axis i goes to bit dim*b + i."""
    k = 0
    for b in range(bits):
        for i in range(dim):
            k |= ((int(q[i]) >> b) & 1) << (dim * b + i)
    return k


@pytest.mark.parametrize("dim,N,p", [(2, 7, 2), (3, 4, 1)])
def test_morton_order_matches_definition(fe, dim, N, p):
    m = shuffled_mesh(structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=3), 11)
    perm = fe.ordering.morton_cell_order(dim, m.coords, m.cell2vertex)
    cen = m.coords[m.cell2vertex].mean(axis=1)
    lo, hi = cen.min(axis=0), cen.max(axis=0)
    bits = 21 if dim == 3 else 32
    levels = (1 << bits) - 1
    q = np.rint(np.clip((cen - lo) / (hi - lo), 0, 1) * levels).astype(np.int64)
    keys = [(_morton_key(q[c], dim, bits), c) for c in range(m.n_cells)]
    assert perm.tolist() == [c for _, c in sorted(keys)]


def test_first_touch_matches_definition(fe):
    m = shuffled_mesh(structured_mesh(3, 3, 2, jitter=0.15, seed=4), 12)
    rng = np.random.default_rng(0)
    order = rng.permutation(m.n_cells).astype(np.int32)
    got = fe.ordering.first_touch_numbering(m.n_nodes + 5, m.cell2node, order)   # 5 unreferenced
    want, nxt = {}, 0
    for c in order:
        for e in m.cell2node[c]:
            if int(e) not in want:
                want[int(e)] = nxt
                nxt += 1
    for e in range(m.n_nodes, m.n_nodes + 5):
        want[e] = nxt
        nxt += 1
    assert got.tolist() == [want[e] for e in range(m.n_nodes + 5)]
    assert np.array_equal(fe.ordering.first_touch_numbering(m.n_nodes, m.cell2node),
                          fe.ordering.first_touch_numbering(m.n_nodes, m.cell2node,
                                                            np.arange(m.n_cells)))


def test_orderings_reject_bad_input(fe):
    m = structured_mesh(2, 3, 1, seed=1)
    bad = m.cell2vertex.copy()
    bad[2, 1] = m.n_vertices
    with pytest.raises(fe.FeError) as e:
        fe.ordering.morton_cell_order(2, m.coords, bad)
    assert e.value.code == 5   # FE_ERR_INDEX
    with pytest.raises(fe.FeError) as e:
        fe.ordering.first_touch_numbering(m.n_nodes, m.cell2node, np.zeros(m.n_cells))
    assert e.value.code == 1   # not a permutation
    nan = m.coords.copy()
    nan[0, 0] = np.nan
    with pytest.raises(fe.FeError):
        fe.ordering.morton_cell_order(2, nan, m.cell2vertex)


def _lines(c2e, group=32, line=8):
    """Mean number of distinct 8-entity blocks (a 64-byte line of doubles) that the
    entities of each group of 32 consecutive cells (a warp) fall into."""
    g = c2e[: (len(c2e) // group) * group].reshape(-1, group * c2e.shape[1]) // line
    return float(np.mean([np.unique(r).size for r in g]))


@pytest.mark.parametrize("dim,N,p", [(2, 40, 2), (3, 12, 1), (3, 8, 2)])
def test_reordering_restores_locality(fe, dim, N, p):
    """A randomly numbered mesh gathers each warp's DoFs from lines all over the
    vector; after the Morton + first-touch ordering a warp's nodes and vertices
    fall into a few lines again, close to the structured numbering."""
    m0 = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=5)
    m = shuffled_mesh(m0, 13)
    perm, vnew, nnew = fe.mesh_order(dim, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    _, c2v, c2n = fe.apply_mesh_order(m.coords, m.cell2vertex, m.cell2node, perm, vnew, nnew)
    assert _lines(c2n) < 0.2 * _lines(m.cell2node)
    assert _lines(c2n) < 1.5 * _lines(m0.cell2node)
    assert _lines(c2v) < 0.2 * _lines(m.cell2vertex)


@pytest.mark.parametrize("kind,dim,N,p,q", [("mass", 2, 6, 3, 6), ("elasticity", 3, 3, 2, 2),
                                            ("laplace", 3, 3, 2, 2)])
def test_reordered_operator_is_the_renumbered_operator(fe, kind, dim, N, p, q):
    m = shuffled_mesh(structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=6), 14)
    perm, vnew, nnew = fe.mesh_order(dim, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    x2, c2v, c2n = fe.apply_mesh_order(m.coords, m.cell2vertex, m.cell2node, perm, vnew, nnew)
    nc = dim if kind == "elasticity" else 1
    u = uniform_field(m.n_nodes * nc, 15)
    o1 = oracle.Oracle(dim, p, q, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o2 = oracle.Oracle(dim, p, q, x2, c2v, c2n, m.n_nodes)
    if kind == "elasticity":
        y1 = o1.elasticity(u, 1.25, 1.0)
        y2 = o2.elasticity(fe.permute_dofs(u, nnew, nc), 1.25, 1.0)
    else:
        y1 = getattr(o1, kind)(u)
        y2 = getattr(o2, kind)(fe.permute_dofs(u, nnew, nc))
    back = fe.unpermute_dofs(y2, nnew, nc)
    assert np.abs(back - y1).max() <= 1e-13 * np.abs(y1).max()
    assert np.array_equal(fe.unpermute_dofs(fe.permute_dofs(u, nnew, nc), nnew, nc), u)
