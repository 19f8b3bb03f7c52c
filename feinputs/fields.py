"""Seeded nodal fields for the synthetic workloads.

All generators use ``numpy.random.Generator(numpy.random.PCG64(seed))``.

* ``uniform_field``: DoF values uniform in [-1, 1] (the mass / elasticity inputs).
* ``sinusoid_displacement``: ``u_c(x) = A * sum_{m=1..M} sin(k_m . x + phi_{m,c})``
  interpolated at the P_p nodes, with angular wave vectors of magnitude in
  [0.5, kmax] and uniform random direction and phases.  With A = 0.05, M = 8 and
  kmax = 1.5 the Frobenius norm of grad u is at most A*M*kmax*sqrt(d) < 1 in 2D,
  so det(I + grad u) > 0 everywhere (the hyperelastic workload's displacement).
* ``lame_fields``: per-cell P0 mu, lambda, log-uniform in the given ranges.
"""

from __future__ import annotations

import numpy as np

from .mesh import SimplexMesh, local_multi_indices


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_field(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """``n`` float64 values uniform in [lo, hi]."""
    return _rng(seed).uniform(lo, hi, size=n)


def node_positions(mesh: SimplexMesh) -> np.ndarray:
    """Physical position of every P_p node, ``[n_nodes, dim]``.

    A node's position is the image of its reference lattice point alpha/p under
    the affine vertex map of any cell containing it (all such cells agree).
    """
    alphas = local_multi_indices(mesh.dim, mesh.degree).astype(np.float64) / mesh.degree
    X = mesh.coords[mesh.cell2vertex]                  # [nc, d+1, d]
    E = X[:, 1:, :] - X[:, :1, :]                      # [nc, d, d]  rows: edge k
    pos = X[:, :1, :] + np.einsum("jk,ckx->cjx", alphas, E)
    out = np.zeros((mesh.n_nodes, mesh.dim))
    out[mesh.cell2node.reshape(-1)] = pos.reshape(-1, mesh.dim)
    return out


def interpolate_at_nodes(mesh: SimplexMesh, fn) -> np.ndarray:
    """Nodal interpolant of ``fn(x[n, d]) -> [n, ncomp]`` flattened ``[node][comp]``."""
    vals = np.asarray(fn(node_positions(mesh)), dtype=np.float64)
    return np.ascontiguousarray(vals.reshape(-1))


def sinusoid_displacement(mesh: SimplexMesh, seed: int, amplitude: float = 0.05,
                          n_modes: int = 8, kmax: float = 1.5) -> np.ndarray:
    """Sum-of-sinusoids displacement interpolated at nodes, ``[n_nodes * dim]``."""
    rng = _rng(seed)
    d = mesh.dim
    mag = rng.uniform(0.5, kmax, size=n_modes)
    dirs = rng.normal(size=(n_modes, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    k = dirs * mag[:, None]                              # [M, d]
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(n_modes, d))   # [M, comp]

    def fn(x):
        arg = x @ k.T                                    # [n, M]
        return amplitude * np.stack(
            [np.sin(arg + phase[None, :, c]).sum(axis=1) for c in range(d)], axis=1)

    return interpolate_at_nodes(mesh, fn)


def lame_fields(n_cells: int, seed: int, mu_range=(0.5, 2.0),
                lam_range=(1.0, 10.0)) -> tuple[np.ndarray, np.ndarray]:
    """Per-cell (mu, lambda), each log-uniform in its range."""
    rng = _rng(seed)
    mu = np.exp(rng.uniform(np.log(mu_range[0]), np.log(mu_range[1]), size=n_cells))
    lam = np.exp(rng.uniform(np.log(lam_range[0]), np.log(lam_range[1]), size=n_cells))
    return mu, lam
