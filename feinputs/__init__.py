"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle's tests.

This package generates *inputs* only: structured simplex meshes of the unit square
and unit cube with jittered interior vertices, the P_p node numbering on the
refined lattice, and seeded coefficient/displacement fields.  It performs none of
the finite element action's arithmetic (no quadrature, no basis functions, no
geometry maps, no forms), so both the library under test and the CPU oracle can
consume its output without sharing any of the method's code.

The workloads follow the paper's experimental setup (Sec. "Experimental Setup"):
meshes of the unit square and the unit cube, with interior vertices jittered by
a seeded generator.  :func:`shuffled_mesh` renumbers a mesh at random (cells,
vertices and nodes), standing in for an unstructured mesh whose numbering
carries no locality.
"""

from .mesh import SimplexMesh, structured_mesh, shuffled_mesh, local_multi_indices, n_local_nodes
from .fields import (uniform_field, sinusoid_displacement, lame_fields,
                     interpolate_at_nodes)

__all__ = [
    "SimplexMesh", "structured_mesh", "shuffled_mesh", "local_multi_indices", "n_local_nodes",
    "uniform_field", "sinusoid_displacement", "lame_fields", "interpolate_at_nodes",
]
