"""Seeded specification of the batched workload: many independent meshes of
uneven size, form and degree.

Each problem: form uniform in {mass, elasticity, neo_hookean}, dimension in
{2, 3}, degree in {1..4}, cell count log-uniform in [cells_min, cells_max]
realised by the structured mesh whose cell count is closest (2 N^2 triangles or
6 N^3 tetrahedra, N >= 1).  Quadrature degree: 2p for mass and Neo-Hookean,
max(2(p-1), 0) for elasticity.  Inputs: u ~ U[-1, 1] for mass and elasticity;
the Neo-Hookean problems use the sum-of-sinusoids displacement (a uniform
[-1, 1] nodal field would invert cells).
"""

from __future__ import annotations

import math

import numpy as np

FORMS = ("mass", "elasticity", "neo_hookean")


def batch_specs(count: int = 64, seed: int = 20250621, cells_min: float = 1e3,
                cells_max: float = 2e5) -> list[dict]:
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        form = FORMS[int(rng.integers(0, 3))]
        dim = int(rng.integers(2, 4))
        degree = int(rng.integers(1, 5))
        cells = math.exp(rng.uniform(math.log(cells_min), math.log(cells_max)))
        if dim == 2:
            N = max(1, round(math.sqrt(cells / 2.0)))
        else:
            N = max(1, round((cells / 6.0) ** (1.0 / 3.0)))
        q = 2 * degree if form != "elasticity" else max(2 * (degree - 1), 0)
        specs.append({"index": i, "form": form, "dim": dim, "degree": degree, "N": N,
                      "quad_degree": q, "seed": seed + 1000 + i,
                      "n_cells": 2 * N * N if dim == 2 else 6 * N ** 3})
    return specs
