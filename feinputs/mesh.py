"""Structured simplex meshes of the unit square / unit cube with seeded jitter.

Conventions (shared layout conventions, not arithmetic of the method):

* Reference simplex: vertices 0, e_1, ..., e_d.
* A cell's vertex list ``cell2vertex[c] = (v_0, ..., v_d)`` defines the affine map
  ``x = x_{v_0} + sum_k xhat_k (x_{v_k} - x_{v_0})``.
* Local P_p nodes are the multi-indices ``alpha = (alpha_1..alpha_d)`` with
  ``alpha_k >= 0`` and ``sum alpha_k <= p``, enumerated by nested loops with
  ``alpha_1`` outermost and ``alpha_d`` innermost, each ascending.  Node ``alpha``
  sits at reference point ``alpha / p``.
* Global P_p nodes live on the ``(p*N + 1)^d`` lattice that refines the vertex
  lattice ``p`` times; the node at lattice point ``(I_1..I_d)`` has id
  ``I_1 + (pN+1) I_2 + (pN+1)^2 I_3`` (x fastest).  Vector fields interleave
  components: DoF ``node * d + comp``.

Cells (Sec. "Experimental Setup": unit square / unit cube domains):

* 2D: every square ``(i, j)`` is split along its diagonal from ``(i, j)`` to
  ``(i+1, j+1)`` into ``[(i,j),(i+1,j),(i+1,j+1)]`` and ``[(i,j),(i+1,j+1),(i,j+1)]``.
* 3D: every cube is split into the 6 Kuhn tetrahedra along its main diagonal;
  vertex order is fixed so that every cell is positively oriented.
* Only interior vertices are jittered, each coordinate independently uniform in
  ``[-a h, a h]`` drawn from ``numpy.random.Generator(PCG64(seed))``; the domain
  stays exactly the unit square / cube.
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from math import comb

import numpy as np


def n_local_nodes(dim: int, degree: int) -> int:
    """Number of P_degree Lagrange nodes on a dim-simplex, C(degree + dim, dim)."""
    return comb(degree + dim, dim)


def local_multi_indices(dim: int, degree: int) -> np.ndarray:
    """Local node multi-indices ``[n_loc, dim]`` in the documented nested-loop order."""
    out = []

    def rec(prefix, remaining, k):
        if k == dim:
            out.append(tuple(prefix))
            return
        for a in range(remaining + 1):
            rec(prefix + [a], remaining - a, k + 1)

    rec([], degree, 0)
    return np.asarray(out, dtype=np.int64)


@dataclass
class SimplexMesh:
    dim: int
    degree: int
    N: int
    coords: np.ndarray        # float64 [n_vertices, dim]
    cell2vertex: np.ndarray   # int32   [n_cells, dim+1]
    cell2node: np.ndarray     # int32   [n_cells, n_loc]
    n_nodes: int
    node_lattice: np.ndarray  # int64   [n_nodes, dim]   lattice coordinates in [0, pN]
    seed: int = 0
    jitter: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.cell2vertex.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_loc(self) -> int:
        return int(self.cell2node.shape[1])

    def boundary_nodes(self) -> np.ndarray:
        """Boolean mask [n_nodes]: node lies on the boundary of the unit square/cube."""
        pn = self.degree * self.N
        return np.any((self.node_lattice == 0) | (self.node_lattice == pn), axis=1)

    def n_dofs(self, n_comp: int) -> int:
        return self.n_nodes * n_comp


def _vertex_id(idx, n1, dim):
    """Vertex lattice index (x fastest) for integer coordinate arrays idx[..., dim]."""
    vid = idx[..., 0].astype(np.int64)
    stride = n1
    for k in range(1, dim):
        vid = vid + stride * idx[..., k]
        stride *= n1
    return vid


def _lattice_points(n: int, dim: int) -> np.ndarray:
    """All integer points of {0..n-1}^dim as ``[n^dim, dim]``, x fastest."""
    idx = np.indices((n,) * dim).reshape(dim, -1)   # idx[k] varies slowest for k=0
    return np.ascontiguousarray(idx[::-1].T)         # column 0 = fastest-varying index


def _cell_templates(dim: int) -> np.ndarray:
    """Unit-cube corner offsets of each sub-simplex, ``[n_sub, dim+1, dim]``."""
    if dim == 2:
        return np.array([[[0, 0], [1, 0], [1, 1]],
                         [[0, 0], [1, 1], [0, 1]]], dtype=np.int64)
    if dim == 3:
        tets = []
        for perm in itertools.permutations(range(3)):
            e = np.eye(3, dtype=np.int64)
            v0 = np.zeros(3, dtype=np.int64)
            v1 = e[perm[0]]
            v2 = e[perm[0]] + e[perm[1]]
            v3 = np.ones(3, dtype=np.int64)
            # orientation of (v1-v0, v2-v0, v3-v0) equals the permutation's sign
            sign = round(np.linalg.det(np.stack([v1, v2, v3], axis=1).astype(float)))
            if sign < 0:
                v1, v2 = v2, v1
            tets.append([v0, v1, v2, v3])
        return np.array(tets, dtype=np.int64)
    raise ValueError("dim must be 2 or 3")


def structured_mesh(dim: int, N: int, degree: int, jitter: float = 0.0,
                    seed: int = 0) -> SimplexMesh:
    """Unit square/cube cut into N^dim squares/cubes, each split into simplices.

    ``jitter`` is the fraction ``a`` of h = 1/N by which interior vertices move
    (uniform in [-a h, a h] per coordinate).  The seeded generator is
    ``numpy.random.Generator(numpy.random.PCG64(seed))``.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if N < 1 or degree < 1:
        raise ValueError("N and degree must be >= 1")
    n1 = N + 1
    h = 1.0 / N

    # vertices ------------------------------------------------------------
    vidx = _lattice_points(n1, dim)
    # vidx[v] = integer coords of vertex v, with v = x + n1*y (+ n1^2*z)
    assert np.array_equal(_vertex_id(vidx, n1, dim), np.arange(vidx.shape[0]))
    coords = vidx.astype(np.float64) * h
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        interior = np.all((vidx > 0) & (vidx < N), axis=1)
        disp = rng.uniform(-jitter * h, jitter * h, size=coords.shape)
        coords = coords + disp * interior[:, None]

    # cells ---------------------------------------------------------------
    tmpl = _cell_templates(dim)                         # [n_sub, dim+1, dim]
    corner = _lattice_points(N, dim)
    # cell vertex integer coords: [n_cubes, n_sub, dim+1, dim]
    cv = corner[:, None, None, :] + tmpl[None, :, :, :]
    cv = cv.reshape(-1, dim + 1, dim)
    cell2vertex = _vertex_id(cv, n1, dim).astype(np.int32)

    # P_p nodes on the p-refined lattice ------------------------------------
    alphas = local_multi_indices(dim, degree)           # [n_loc, dim]
    v0 = cv[:, 0, :]                                    # [nc, dim]
    edges = cv[:, 1:, :] - v0[:, None, :]               # [nc, dim(k), dim(coord)]
    # lattice point of local node alpha: p*v0 + sum_k alpha_k (v_k - v0)
    lat = degree * v0[:, None, :] + np.einsum("jk,ckx->cjx", alphas, edges)
    pn1 = degree * N + 1
    cell2node = _vertex_id(lat, pn1, dim).astype(np.int64)
    n_nodes = pn1 ** dim
    node_lattice = np.zeros((n_nodes, dim), dtype=np.int64)
    node_lattice[cell2node.reshape(-1)] = lat.reshape(-1, dim)

    if n_nodes * max(dim, 1) >= 2 ** 31:
        raise ValueError("mesh too large for int32 DoF indices")

    return SimplexMesh(dim=dim, degree=degree, N=N, coords=np.ascontiguousarray(coords),
                       cell2vertex=np.ascontiguousarray(cell2vertex),
                       cell2node=np.ascontiguousarray(cell2node.astype(np.int32)),
                       n_nodes=int(n_nodes), node_lattice=node_lattice,
                       seed=seed, jitter=jitter, meta={"h": h})


def shuffled_mesh(mesh: SimplexMesh, seed: int) -> SimplexMesh:
    """The same mesh with its cells, vertices and nodes renumbered by seeded
    random permutations: an unstructured numbering with no locality.  Node k of
    the result is node ``meta["node_old"][k]`` of ``mesh``; cell k is cell
    ``meta["cell_old"][k]``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cell_old = rng.permutation(mesh.n_cells)
    vert_old = rng.permutation(mesh.n_vertices)
    node_old = rng.permutation(mesh.n_nodes)
    vert_new = np.empty_like(vert_old)
    vert_new[vert_old] = np.arange(vert_old.size)
    node_new = np.empty_like(node_old)
    node_new[node_old] = np.arange(node_old.size)
    return SimplexMesh(dim=mesh.dim, degree=mesh.degree, N=mesh.N,
                       coords=np.ascontiguousarray(mesh.coords[vert_old]),
                       cell2vertex=np.ascontiguousarray(vert_new[mesh.cell2vertex[cell_old]].astype(np.int32)),
                       cell2node=np.ascontiguousarray(node_new[mesh.cell2node[cell_old]].astype(np.int32)),
                       n_nodes=mesh.n_nodes, node_lattice=mesh.node_lattice[node_old],
                       seed=mesh.seed, jitter=mesh.jitter,
                       meta=dict(mesh.meta, cell_old=cell_old, node_old=node_old, vert_old=vert_old))
