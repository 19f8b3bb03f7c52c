"""Structural zeros of the reference gradient tables.

The basis function of barycentric multi-index alpha depends on lam_0 = 1 - sum
xhat only through alpha_0 and on lam_k = xhat_k only through alpha_k, so its
derivative d/dxhat_k vanishes identically when alpha_0 = alpha_k = 0.  The
thread-per-cell kernels skip those table entries and the algorithmic flop count
leaves them out.  Pinned here without a GPU:
  * in the oracle's independent tabulation those entries are zero to rounding at
    every point, and every other entry is nonzero somewhere (the rule is exact
    and complete);
  * the library's tabulation holds exactly 0.0 there (a fused multiply-add with
    that factor returns its addend, so skipping changes no result);
  * fe_action_noalloc refuses a caller table that breaks a structural zero,
    before any device work.
The GPU test checks the plans' flop counts against the same rule."""

import ctypes
from math import comb

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2506_17471_gb300 as fe
    return fe


def multi_indices(dim, p):
    """(alpha_0, alpha_1, ..., alpha_d) of each local node, alpha_1 outermost."""
    out = []
    if dim == 2:
        for a in range(p + 1):
            for b in range(p + 1 - a):
                out.append((p - a - b, a, b))
    else:
        for a in range(p + 1):
            for b in range(p + 1 - a):
                for c in range(p + 1 - a - b):
                    out.append((p - a - b - c, a, b, c))
    return out


def zero_pattern(dim, p):
    """Boolean [dim, n]: True where d phi_j / dxhat_k vanishes identically."""
    al = multi_indices(dim, p)
    return np.array([[a[0] == 0 and a[k + 1] == 0 for a in al] for k in range(dim)])


def nonzero_count(dim, p):
    return dim * comb(p + dim, dim) - int(zero_pattern(dim, p).sum())


CASES = [(2, p) for p in range(1, 9)] + [(3, p) for p in range(1, 7)]


@pytest.mark.parametrize("dim,p", CASES)
def test_rule_is_exact_and_complete_on_the_oracle_tables(dim, p):
    import oracle
    _, _, t = oracle.tabulate(dim, p, 2 * p)
    z = zero_pattern(dim, p)
    grads = np.abs(t[1:])                       # [dim, nq, n]
    scale = grads.max()
    peak = grads.max(axis=1)                    # [dim, n]: largest |entry| over the points
    assert np.all(peak[z] <= 1e-13 * scale)
    assert np.all(peak[~z] > 1e-6 * scale)


def test_zero_counts_by_hand():
    # P1 tetrahedron: the three vertices off the origin have one nonzero derivative each
    assert zero_pattern(3, 1).sum() == 6 and nonzero_count(3, 1) == 6
    # P2 tetrahedron: 3 vertex functions x 2 zeros + 3 edge functions x 1 zero
    assert zero_pattern(3, 2).sum() == 9 and nonzero_count(3, 2) == 21
    # P2 triangle: the two vertex functions off the origin, one zero each
    assert zero_pattern(2, 2).sum() == 2 and nonzero_count(2, 2) == 10


@pytest.mark.parametrize("dim,p", CASES)
@pytest.mark.parametrize("scheme", ["conical", "symmetric"])
def test_library_tables_hold_exact_zeros(fe, dim, p, scheme):
    _, _, t = fe.tabulate(dim, p, 2 * p, scheme)
    z = zero_pattern(dim, p)
    for k in range(dim):
        assert np.all(t[1 + k][:, z[k]] == 0.0)


def test_noalloc_refuses_a_table_that_breaks_a_structural_zero(fe):
    """The host check runs before any device call, so fake device pointers are
    never dereferenced; the same call with the true table passes that check and
    only then fails at the device query (no GPU here) or runs (on a GPU)."""
    from paper_2506_17471_gb300 import _native as N
    fake = ctypes.c_void_p(0x10000)
    _, wts, tab = fe.tabulate(3, 2, 2, "symmetric")
    tab, wts = np.ascontiguousarray(tab), np.ascontiguousarray(wts)
    j = int(np.flatnonzero(zero_pattern(3, 2)[0])[0])
    bad = tab.copy()
    bad[1, 0, j] = 1e-300

    def call(t):
        mesh = N.FeMesh(3, 2, 64, 6, 125, fake, fake, fake)
        form = N.FeForm(N.FE_FORM_ELASTICITY, 2, N.FE_PREC_FP64, 0, 1.25, 1.0, None, None, None, 0, 0)
        return N.lib.fe_action_noalloc(ctypes.byref(form), ctypes.byref(mesh),
                                       t.ctypes.data_as(ctypes.c_void_p),
                                       wts.ctypes.data_as(ctypes.c_void_p), int(len(wts)),
                                       fake, ctypes.c_void_p(0x20000), None, None)

    assert call(bad) == N.FE_ERR_INVALID_ARG
    import torch
    if not torch.cuda.is_available():
        assert call(tab) == N.FE_ERR_CUDA


@pytest.mark.gpu
@pytest.mark.parametrize("kind,dim,p,q", [("ELASTICITY", 3, 2, 2), ("ELASTICITY", 2, 2, 2),
                                          ("NH_JACOBIAN", 3, 1, 2), ("LAPLACE", 3, 3, 4),
                                          ("HELMHOLTZ", 2, 4, 8), ("MASS", 3, 2, 4)])
def test_plan_flop_counts_follow_the_rule(fe, kind, dim, p, q):
    """flops_per_cell_dense - flops_per_cell = the skipped multiply-adds: per
    point, 2 flops x (field evaluations + one test contraction) x components x
    structural zeros."""
    import torch
    from feinputs import structured_mesh
    m = structured_mesh(dim, 2, p, seed=1)
    mesh = fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    nc = dim if kind in ("ELASTICITY", "NH_JACOBIAN") else 1
    kw = {}
    if kind == "NH_JACOBIAN":
        kw["u_lin"] = torch.zeros(m.n_nodes * nc, dtype=torch.float64, device="cuda")
    plan = fe.Plan(mesh, getattr(fe, kind), q, lam=1.25, mu=1.0, **kw)
    zeros = int(zero_pattern(dim, p).sum())
    contractions = {"ELASTICITY": 2, "NH_JACOBIAN": 3, "LAPLACE": 2, "HELMHOLTZ": 2, "MASS": 0}[kind]
    gap = plan.info.flops_per_cell_dense - plan.info.flops_per_cell
    assert gap == plan.info.nq * 2 * contractions * nc * zeros
