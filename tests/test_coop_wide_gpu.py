"""Edge cases of the cells-per-CTA kernel's wide layout (FP64 gradient forms on
tetrahedra: one 512-thread CTA per SM as two independent 256-thread groups, each
with its own 32-cell batches, named barrier and batch scratch behind a shared
table; node-major quadrature phase that skips the structurally zero directions).

Cases: batch boundaries (1, 63, 64, 65, 129 cells), meshes with fewer units than
CTAs and with many units per CTA, the last partial round of units split by
quadrature points, the accumulate flag, out-of-range indices and a
degenerate cell in the middle of a batch (the rest of the batch is still applied),
and the Neo-Hookean adjoint (per-cell material derivatives) on a ragged batch.
"""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_17471_gb300 as fe
    return fe


def rel(a, b):
    a = a.detach().cpu().numpy() if torch.is_tensor(a) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sub(fe, m, cells):
    M = fe.Mesh(3, m.degree, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes)
    o = oracle.Oracle(3, m.degree, 6, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes, "symmetric")
    return M, o


def wide_plan(fe, M, **kw):
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, quad_scheme="symmetric", **kw)
    assert plan.info.kernel == 1 and plan.info.threads_per_block == 512
    return plan


@pytest.mark.parametrize("n_cells", [1, 63, 64, 65, 129])
def test_wide_layout_batch_boundaries(fe, n_cells):
    m = structured_mesh(3, 3, 4, jitter=0.15, seed=600)
    M, o = sub(fe, m, np.arange(n_cells))
    u = uniform_field(m.n_nodes * 3, 601)
    plan = wide_plan(fe, M)
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL
    assert plan.status() == 0


@pytest.mark.parametrize("N", [6, 11])
def test_wide_layout_units_per_cta(fe, N):
    """N=6: 1,296 cells, 41 units for 152 CTAs (some groups get none); N=11:
    7,986 cells, 250 units for 304 groups."""
    m = structured_mesh(3, N, 4, jitter=0.15, seed=610 + N)
    M = fe.Mesh(3, 4, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 6, "symmetric")
    u = uniform_field(m.n_nodes * 3, 611)
    plan = wide_plan(fe, M)
    y = plan.apply(cuda(u))
    assert rel(y, o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    # repeated launches reuse the self-resetting queue counters
    y2 = plan.apply(cuda(u))
    assert rel(y2, y.cpu().numpy()) <= 1e-15
    assert plan.status() == 0


def test_wide_layout_tail_split(fe):
    """17^3 x 6 = 29,478 cells, 922 32-cell units (the last one ragged) for 304
    groups: three full rounds, then a tail of 10 units that the kernel hands out as
    10 x 24 items of one quadrature point each, every item adding its part of the
    quadrature sum through the same scatter.  Elasticity and the Neo-Hookean
    residual and Jacobian action against the oracle, and the accumulate flag."""
    m = structured_mesh(3, 17, 4, jitter=0.15, seed=615)
    M = fe.Mesh(3, 4, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 6, "symmetric")
    u = uniform_field(m.n_nodes * 3, 616)
    plan = wide_plan(fe, M)
    assert plan.info.grid_blocks == 152
    y = plan.apply(cuda(u))
    assert rel(y, o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    y0 = uniform_field(m.n_nodes * 3, 617)
    acc = wide_plan(fe, M, accumulate=True)
    assert rel(acc.apply(cuda(u), cuda(y0.copy())), y0 + o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    mu, lam = lame_fields(m.n_cells, 618)
    ud = sinusoid_displacement(m, 619)
    res = fe.Plan(M, fe.NH_RESIDUAL, 6, mu_cell=mu, lam_cell=lam, quad_scheme="symmetric")
    assert res.info.kernel == 1 and res.info.threads_per_block == 512
    assert rel(res.apply(cuda(ud)), o.nh_residual(ud, mu, lam, threads=16)) <= TOL
    jac = fe.Plan(M, fe.NH_JACOBIAN, 6, mu_cell=mu, lam_cell=lam, u_lin=ud, quad_scheme="symmetric")
    assert rel(jac.apply(cuda(u)), o.nh_jacobian(ud, u, mu, lam, threads=16)) <= TOL
    for p in (plan, acc, res, jac):
        assert p.status() == 0


def test_wide_layout_accumulate(fe):
    m = structured_mesh(3, 3, 4, jitter=0.15, seed=620)
    M, o = sub(fe, m, np.arange(m.n_cells))
    u = uniform_field(m.n_nodes * 3, 621)
    y0 = uniform_field(m.n_nodes * 3, 622)
    plan = wide_plan(fe, M, accumulate=True)
    y = plan.apply(cuda(u), cuda(y0.copy()))
    assert rel(y, y0 + o.elasticity(u, 1.25, 1.0)) <= TOL


def test_wide_layout_bad_index_and_degenerate_cell(fe):
    """Cell 40 (inside the first 64-cell batch) has an out-of-range node and cell
    70 (the second batch) is degenerate: both are skipped and reported, every
    other cell of their batches is applied."""
    from paper_2506_17471_gb300 import _native as N
    m = structured_mesh(3, 3, 4, jitter=0.15, seed=630)
    c2n = m.cell2node.copy()
    c2n[40, 17] = m.n_nodes + 3
    M = fe.Mesh(3, 4, m.coords, m.cell2vertex, c2n, m.n_nodes)
    u = uniform_field(m.n_nodes * 3, 631)
    plan = wide_plan(fe, M)
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == N.FE_ERR_INDEX
    keep = np.ones(m.n_cells, dtype=bool)
    keep[40] = False
    _, o = sub(fe, m, np.nonzero(keep)[0])
    assert rel(y, o.elasticity(u, 1.25, 1.0)) <= TOL
    bad = m.cell2vertex.copy()
    bad[70, 3] = bad[70, 0]                                      # cell 70 collapses to a face
    M2 = fe.Mesh(3, 4, m.coords, bad, m.cell2node, m.n_nodes)
    plan2 = wide_plan(fe, M2)
    y2 = plan2.apply(cuda(u)).cpu().numpy()
    assert plan2.status() == N.FE_ERR_BAD_MESH
    keep = np.ones(m.n_cells, dtype=bool)
    keep[70] = False
    _, o2 = sub(fe, m, np.nonzero(keep)[0])
    assert rel(y2, o2.elasticity(u, 1.25, 1.0)) <= TOL


def test_wide_layout_neo_hookean_adjoint(fe):
    """NH residual, Jacobian action and adjoint on P3 tetrahedra (200 cells: three
    full batches and a ragged one)."""
    m = structured_mesh(3, 4, 3, jitter=0.15, seed=640)
    cells = np.arange(200)
    M = fe.Mesh(3, 3, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes)
    o = oracle.Oracle(3, 3, 6, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes, "symmetric")
    mu, lam = lame_fields(200, 641)
    u = sinusoid_displacement(m, 642)
    w = uniform_field(m.n_nodes * 3, 643)
    res = fe.Plan(M, fe.NH_RESIDUAL, 6, mu_cell=mu, lam_cell=lam, quad_scheme="symmetric")
    assert res.info.kernel == 1 and res.info.threads_per_block == 512
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL
    jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, ojtw) <= TOL and rel(dmu, odmu) <= TOL and rel(dlam, odlam) <= TOL
    jac = fe.Plan(M, fe.NH_JACOBIAN, 6, mu_cell=mu, lam_cell=lam, u_lin=cuda(u), quad_scheme="symmetric")
    assert rel(jac.apply(cuda(w)), o.nh_jacobian(u, w, mu, lam)) <= TOL
    assert res.status() == 0 and jac.status() == 0
