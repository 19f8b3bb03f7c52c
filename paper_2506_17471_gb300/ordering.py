"""Locality orderings of a mesh (host side, through ``fe_order_cells_morton`` and
``fe_order_first_touch``).

At low order the action is dominated by its indirect gathers and scatters;
keeping the DoFs of cells processed together close in memory lets them share
cache lines (Sec. "Behavior at low orders").  :func:`mesh_order` computes a
Morton order of the cells and first-touch numberings of vertices and nodes;
:func:`apply_mesh_order` renumbers the mesh arrays; :func:`permute_dofs` and
:func:`unpermute_dofs` move DoF vectors between the two numberings.  The
reordered mesh defines the same operator: y' = A'(u') with u' = P u gives
y' = P y.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def morton_cell_order(dim: int, coords, cell2vertex) -> np.ndarray:
    """Old cell index of each position of the Morton order of the cell centroids."""
    x = np.ascontiguousarray(np.asarray(coords, dtype=np.float64))
    c2v = _i32(cell2vertex)
    n_cells = c2v.shape[0]
    perm = np.empty(n_cells, dtype=np.int32)
    N.check(N.lib.fe_order_cells_morton(int(dim), x.shape[0], n_cells, _p(x), _p(c2v), _p(perm)),
            "fe_order_cells_morton")
    return perm


def first_touch_numbering(n_entities: int, cell2entity, cell_order=None) -> np.ndarray:
    """New index of each entity, numbered as the cells (in ``cell_order``) first use it."""
    c2e = _i32(cell2entity)
    order = None if cell_order is None else _i32(cell_order)
    new_of_old = np.empty(int(n_entities), dtype=np.int32)
    N.check(N.lib.fe_order_first_touch(int(n_entities), c2e.shape[0], c2e.shape[1], _p(c2e),
                                       ctypes.c_void_p(0) if order is None else _p(order), _p(new_of_old)),
            "fe_order_first_touch")
    return new_of_old


def mesh_order(dim: int, coords, cell2vertex, cell2node, n_nodes: int):
    """(cell_perm, vertex_new_of_old, node_new_of_old): Morton cell order, then
    vertices and nodes numbered by first touch in that order."""
    perm = morton_cell_order(dim, coords, cell2vertex)
    vnew = first_touch_numbering(np.asarray(coords).shape[0], cell2vertex, perm)
    nnew = first_touch_numbering(n_nodes, cell2node, perm)
    return perm, vnew, nnew


def apply_mesh_order(coords, cell2vertex, cell2node, cell_perm, vertex_new_of_old, node_new_of_old):
    """(coords', cell2vertex', cell2node') of the renumbered mesh: new cell k is old
    cell ``cell_perm[k]``; entity indices are mapped through the new-of-old arrays."""
    x = np.asarray(coords, dtype=np.float64)
    vnew = np.asarray(vertex_new_of_old)
    coords2 = np.empty_like(x)
    coords2[vnew] = x
    c2v = np.asarray(vertex_new_of_old)[np.asarray(cell2vertex)[cell_perm]].astype(np.int32)
    c2n = np.asarray(node_new_of_old)[np.asarray(cell2node)[cell_perm]].astype(np.int32)
    return coords2, np.ascontiguousarray(c2v), np.ascontiguousarray(c2n)


def permute_dofs(u, node_new_of_old, ncomp: int) -> np.ndarray:
    """u' with u'[new(i) * ncomp + c] = u[i * ncomp + c] (interleaved DoFs)."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, ncomp)
    out = np.empty_like(u)
    out[np.asarray(node_new_of_old)] = u
    return out.reshape(-1)


def unpermute_dofs(v, node_new_of_old, ncomp: int) -> np.ndarray:
    """The inverse of :func:`permute_dofs`."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, ncomp)
    return v[np.asarray(node_new_of_old)].reshape(-1)
