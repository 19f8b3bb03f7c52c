"""GPU tests of the node-gather scatter (FE_FLAG_GATHER_SCATTER): per-cell outputs
stored, then summed per node in the fixed order of the incidence list.  Same
results as the atomic scatter (FP64: to 1e-12 of the oracle), bitwise identical
across runs, through every kernel and precision."""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 5e-5), ("fp16", 8 * 2.0 ** -11)])
@pytest.mark.parametrize("coop", [False, True])
def test_gather_scatter_elasticity(fe, prec, tol, coop):
    if coop and prec == "fp16":
        pytest.skip("the 16-bit precisions have one kernel")
    m = structured_mesh(3, 5, 2, jitter=0.15, seed=91)
    M = fe.Mesh(3, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 2)
    u = uniform_field(m.n_nodes * 3, 92)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0, precision=prec, cooperative=coop, gather_scatter=True)
    y1 = plan.apply(cuda(u))
    y2 = plan.apply(cuda(u))
    assert torch.equal(y1, y2)                      # deterministic
    assert rel(y1, o.elasticity(u, 1.25, 1.0)) <= tol
    assert plan.status() == 0


def test_gather_scatter_forms_and_accumulate(fe):
    m = structured_mesh(2, 13, 4, jitter=0.2, seed=93)
    M = fe.Mesh(2, 4, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 94)
    ul = sinusoid_displacement(m, 95)
    du = uniform_field(m.n_nodes * 2, 96)
    jac = fe.Plan(M, fe.NH_JACOBIAN, 8, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), gather_scatter=True)
    assert rel(jac.apply(cuda(du)), o.nh_jacobian(ul, du, mu, lam)) <= 1e-12
    us = uniform_field(m.n_nodes, 97)
    y0 = uniform_field(m.n_nodes, 98)
    hel = fe.Plan(M, fe.HELMHOLTZ, 8, accumulate=True, gather_scatter=True)
    y = hel.apply(cuda(us), cuda(y0.copy()))
    assert rel(y, y0 + o.helmholtz(us)) <= 1e-12
    tc = fe.Plan(M, fe.NH_JACOBIAN, 8, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision="bf16",
                 gather_scatter=True)
    a, b = tc.apply(cuda(du)), tc.apply(cuda(du))
    assert torch.equal(a, b) and rel(a, o.nh_jacobian(ul, du, mu, lam)) <= 8 * 2.0 ** -8
    # the adjoint keeps its atomic scatter and agrees with the plain plan
    res = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam, gather_scatter=True)
    jtw, dmu, dlam = res.adjoint(cuda(ul), cuda(du))
    ojtw, odmu, odlam = o.nh_adjoint(ul, du, mu, lam)
    assert rel(jtw, ojtw) <= 1e-12
    assert jac.status() == 0 and hel.status() == 0 and tc.status() == 0 and res.status() == 0


def test_gather_scatter_skips_bad_cells(fe):
    """A cell with an out-of-range node index contributes nothing (its stored
    outputs are zeros, even after a call with a valid mesh filled the buffer)."""
    from paper_2506_17471_gb300 import _native as N
    m = structured_mesh(2, 13, 3, jitter=0.2, seed=99)
    c2n = m.cell2node.copy()
    c2n[77, 3] = m.n_nodes + 5
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex, c2n, m.n_nodes)
    plan = fe.Plan(M, fe.MASS, 6, gather_scatter=True)
    u = uniform_field(m.n_nodes, 100)
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == N.FE_ERR_INDEX
    keep = np.ones(m.n_cells, dtype=bool)
    keep[77] = False
    o = oracle.Oracle(2, 3, 6, m.coords, m.cell2vertex[keep], m.cell2node[keep], m.n_nodes)
    assert rel(y, o.mass(u)) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp16", 8 * 2.0 ** -11), ("fp16x2", 5e-5), ("tf32", 8 * 2.0 ** -11)])
def test_gather_scatter_tensor_cores_threads_per_cell(fe, prec, tol):
    """Elasticity P4 3D on the tensor cores runs two pipelines (FP16) or one (split
    FP16, TF32), each with two threads per cell; the per-cell stores of the
    deterministic scatter are split among the cell's threads."""
    m = structured_mesh(3, 4, 4, jitter=0.15, seed=93)
    M = fe.Mesh(3, 4, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 6)
    u = uniform_field(m.n_nodes * 3, 94)
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, precision=prec, gather_scatter=True)
    assert plan.info.kernel == 2 and plan.info.threads_per_block == (512 if prec == "fp16" else 256)
    y1 = plan.apply(cuda(u))
    y2 = plan.apply(cuda(u))
    assert torch.equal(y1, y2)
    assert rel(y1, o.elasticity(u, 1.25, 1.0)) <= tol
    assert plan.status() == 0
