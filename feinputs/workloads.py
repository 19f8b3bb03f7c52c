"""Named workloads: the meshes and fields of the benchmark configurations.

Input generation only (sizes, seeds, generators); none of the action's
arithmetic.  Both the benchmark and the tests build their inputs from here, so
a parity test at full size sees exactly the arrays the benchmark times.
"""

from __future__ import annotations

from dataclasses import dataclass

from .fields import uniform_field
from .mesh import structured_mesh


@dataclass(frozen=True)
class ElasticityWorkload:
    """Linear elasticity, vector P_degree on the jittered unit cube (6 Kuhn
    tetrahedra per cube), constant Lame parameters, u ~ U[-1, 1]."""
    name: str
    N: int
    degree: int
    quad_degree: int
    quad_scheme: str
    lam: float = 1.25
    mu: float = 1.0
    jitter: float = 0.15

    @property
    def mesh_seed(self) -> int:
        return 20250620 + self.N

    field_seed: int = 4

    def mesh(self):
        return structured_mesh(3, self.N, self.degree, jitter=self.jitter, seed=self.mesh_seed)

    def field(self, mesh):
        return uniform_field(mesh.n_nodes * 3, self.field_seed)

    def describe(self, mesh, nq: int) -> str:
        return (f"linear elasticity, vector P{self.degree} tets, unit cube {self.N}^3 x 6 Kuhn tets "
                f"({mesh.n_cells:,} cells, {mesh.n_nodes * 3:,} DoFs), jitter {self.jitter}h, "
                f"lambda={self.lam} mu={self.mu}, quadrature degree {self.quad_degree} "
                f"({nq}-point {self.quad_scheme} rule), u~U[-1,1], FP64")


# The hp-sweep point at ~16M DoFs: elasticity P4 on 43^3 x 6 = 477,042 tetrahedra
# (15,533,151 DoFs), quadrature exact to degree 6 = 2(p - 1), the degree of the
# integrand grad u : grad v on affine cells, with the 24-point fully symmetric rule.
ELASTICITY_P4_3D_N43 = ElasticityWorkload("elasticity_p4_3d_n43", N=43, degree=4, quad_degree=6,
                                          quad_scheme="symmetric")
# The same at ~4M DoFs (27^3 x 6 = 118,098 tetrahedra, 3,885,087 DoFs).
ELASTICITY_P4_3D_N27 = ElasticityWorkload("elasticity_p4_3d_n27", N=27, degree=4, quad_degree=6,
                                          quad_scheme="symmetric")
