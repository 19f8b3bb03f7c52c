"""GB300-native matrix-free finite element actions (arXiv 2506.17471's hot path).

y = A(u) for the mass, Laplacian, Helmholtz, linear elasticity, compressible
Neo-Hookean and St. Venant-Kirchhoff forms on affine simplex meshes, computed by
hand-written sm_103a CUDA kernels behind the
C-ABI declared in include/feaction.h.  Importing the package loads the in-tree
shared library and raises ImportError if it has not been built.
"""

from ._native import FeError, LIB_PATH, EXPORTS
from .api import (MASS, ELASTICITY, NH_RESIDUAL, NH_JACOBIAN, LAPLACE, HELMHOLTZ, SVK_RESIDUAL,
                  SVK_JACOBIAN, FORM_NAMES, PRECISIONS, QUAD_SCHEMES,
                  Mesh, Plan,
                  PlanInfo,
                  NeoHookeanResidual, Batch, tabulate, measure_fp64_peak, action)
from .solvers import cg, cg_ir
from .ordering import mesh_order, apply_mesh_order, permute_dofs, unpermute_dofs

__all__ = ["FeError", "LIB_PATH", "EXPORTS", "MASS", "ELASTICITY", "NH_RESIDUAL", "NH_JACOBIAN",
           "LAPLACE", "HELMHOLTZ", "SVK_RESIDUAL", "SVK_JACOBIAN",
           "FORM_NAMES", "PRECISIONS", "QUAD_SCHEMES", "Mesh", "Plan", "PlanInfo", "NeoHookeanResidual", "Batch", "tabulate",
           "measure_fp64_peak", "action", "cg", "cg_ir", "mesh_order", "apply_mesh_order", "permute_dofs",
           "unpermute_dofs"]
