"""Stated accuracy bounds of the reduced-precision actions against the FP64 oracle.

A bound is norm-wise: ||y - y_ref||_inf <= bound * ||y_ref||_inf.  The 16-bit and
TF32 tensor-core paths round three things to 16 significant bits or fewer (the
tables, each cell's scaled DoFs and the scaled pointwise values) and accumulate
in FP32, so their error is a multiple of the unit roundoff u16 (bfloat16 2^-8,
binary16 and TF32 2^-11), the multiple depending on the form: the ratio of the
absolute terms to the result through the two contractions, and for the
Neo-Hookean Jacobian the smooth linearisation point evaluated from 16-bit data.
Each per-form multiple K16 below is the largest deviation measured over the
tensor-core tests of this suite (all degrees, 2D and 3D, hp-sweep sizes, scaled
meshes and materials; MEASURED16, in units of u16) times a margin of 1.5,
rounded up to a quarter (so between 1.25 u16 and 6.5 u16; the earlier uniform
bound was 8 u16).

Tests call :func:`check16`, which also records the deviation when the
environment variable FE_DEVIATION_LOG names a file (written at the end of the
session by tests/conftest.py); that record is how MEASURED16 was obtained.
"""

from __future__ import annotations

import math
import os

U16 = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "tf32": 2.0 ** -11}
FORMS = ("mass", "elasticity", "laplace", "helmholtz", "nh_jacobian", "svk_jacobian")

# largest measured deviation per (form, precision), in units of u16, over this
# suite's tensor-core cases on a GB300 (101 cases; the case that set each maximum
# in the comment).  TF32 carries binary16's significand: where a form has no TF32
# case its binary16 figure stands in.
MEASURED16: dict[tuple[str, str], float] = {
    ("mass", "bf16"): 1.469,          # P3 triangles, 12-point rule
    ("mass", "fp16"): 0.844,          # P3 triangles, 4M DoFs
    ("mass", "tf32"): 0.809,          # P1 triangles
    ("elasticity", "bf16"): 1.180,    # P2 triangles, 3-point rule
    ("elasticity", "fp16"): 1.344,    # P2 triangles, 3-point rule
    ("elasticity", "tf32"): 1.344,    # P2 triangles, 3-point rule
    ("laplace", "bf16"): 1.078,       # P2 triangles
    ("laplace", "fp16"): 0.934,       # P2 triangles
    ("laplace", "tf32"): 0.934,       # (binary16's figure)
    ("helmholtz", "bf16"): 0.854,     # P3 triangles on a mesh scaled by 2^20
    ("helmholtz", "fp16"): 0.916,     # the same
    ("helmholtz", "tf32"): 0.917,     # the same
    ("nh_jacobian", "bf16"): 2.561,   # P6 triangles
    ("nh_jacobian", "fp16"): 4.300,   # P6 triangles, 4M DoFs
    ("nh_jacobian", "tf32"): 3.118,   # P6 triangles
    ("svk_jacobian", "bf16"): 1.078,  # P4 triangles
    ("svk_jacobian", "fp16"): 1.246,  # P4 triangles
    ("svk_jacobian", "tf32"): 1.246,  # P4 triangles
}

MARGIN = 1.5


def k16(form: str, prec: str) -> float:
    return math.ceil(MEASURED16[(form, prec)] * MARGIN * 4.0) / 4.0


def bound16(form: str, prec: str) -> float:
    return k16(form, prec) * U16[prec]


DEVIATIONS: list[dict] = []


def record(form: str, prec: str, err: float, case: str) -> None:
    if os.environ.get("FE_DEVIATION_LOG"):
        DEVIATIONS.append({"form": form, "prec": prec, "err": err, "u16": err / U16[prec] if prec in U16 else None,
                           "case": case})


def check16(form: str, prec: str, err: float, case: str = "", floor: float | None = 1e-7) -> None:
    """Record err and assert it lies within the form's stated bound (and above a
    floor that shows the contractions really ran in reduced precision)."""
    record(form, prec, err, case)
    assert (form, prec) in MEASURED16, (form, prec)
    assert err <= bound16(form, prec), (form, prec, err, bound16(form, prec))
    if floor is not None:
        assert err > floor, (form, prec, err)
