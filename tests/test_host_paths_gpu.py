"""GPU tests of the end-to-end host entry points: fe_action_host (one
synchronous step) and fe_action_host_pipelined (copies and actions of
successive steps overlapped through two device buffer pairs)."""

import ctypes

import numpy as np
import pytest
import torch

from feinputs import structured_mesh, uniform_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_17471_gb300 as fe
    m = structured_mesh(3, 9, 2, jitter=0.15, seed=17)
    M = fe.Mesh(3, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0)
    return fe, m, plan


def test_pipelined_matches_device_action(setup):
    fe, m, plan = setup
    n = m.n_nodes * 3
    us = [torch.from_numpy(uniform_field(n, 100 + i)).pin_memory() for i in range(7)]
    ys = plan.apply_host_pipelined(us)
    for u, y in zip(us, ys):
        ref = plan.apply(u.cuda()).cpu()
        assert torch.equal(y, ref) or float((y - ref).abs().max() / ref.abs().max()) < 1e-14
    # the synchronous single-step path agrees too
    y1 = plan.apply_host(us[3])
    assert float((y1 - ys[3]).abs().max() / ys[3].abs().max()) < 1e-14
    assert plan.status() == 0


def test_pipelined_reused_buffers_and_edge_cases(setup):
    fe, m, plan = setup
    n = m.n_nodes * 3
    pool = [torch.from_numpy(uniform_field(n, 200 + i)).pin_memory() for i in range(2)]
    out = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    # steps cycling through two inputs and two outputs (ordered on the copy streams)
    ys = plan.apply_host_pipelined([pool[i % 2] for i in range(6)], [out[i % 2] for i in range(6)])
    for i in (4, 5):
        ref = plan.apply(pool[i % 2].cuda()).cpu()
        assert float((ys[i] - ref).abs().max() / ref.abs().max()) < 1e-14
    assert plan.apply_host_pipelined([]) == []
    from paper_2506_17471_gb300 import _native as N
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    up = (P * 1)(pool[0].data_ptr())
    yp = (P * 1)(out[0].data_ptr())
    same = (P * 2)(d.data_ptr(), d.data_ptr())
    assert N.lib.fe_action_host_pipelined(plan._h, 1, up, yp, same, same, None) == N.FE_ERR_INVALID_ARG
    assert N.lib.fe_action_host_pipelined(plan._h, -1, up, yp, same, same, None) == N.FE_ERR_INVALID_ARG


def test_one_call_action_caches_plans(setup):
    """fe.action builds each (form, options) plan once, keeps it on the mesh and
    copies per-call fields into it; results equal an explicit plan's."""
    import oracle
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    fe, m, plan = setup
    M = plan.mesh
    u = torch.from_numpy(uniform_field(m.n_nodes * 3, 5)).cuda()
    y = fe.action(M, fe.ELASTICITY, u, 2, lam=1.25, mu=1.0)
    assert torch.equal(y, plan.apply(u)) or float((y - plan.apply(u)).abs().max() / y.abs().max()) < 1e-14
    fe.action(M, fe.ELASTICITY, u, 2, lam=1.25, mu=1.0)
    assert len(M._action_plans) == 1
    # per-cell fields: a second set of coefficients reuses the cached plan
    o = oracle.Oracle.from_mesh(m, 4)
    ul = sinusoid_displacement(m, 3)
    for seed in (1, 2):
        mu, lam = lame_fields(m.n_cells, seed)
        r = fe.action(M, fe.NH_RESIDUAL, torch.from_numpy(ul).cuda(), 4, mu_cell=mu, lam_cell=lam)
        ref = o.nh_residual(ul, mu, lam)
        assert np.abs(r.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert len(M._action_plans) == 2
    # a host input goes through the end-to-end path
    yh = fe.action(M, fe.ELASTICITY, u.cpu(), 2, lam=1.25, mu=1.0)
    assert not yh.is_cuda and float((yh - y.cpu()).abs().max() / y.abs().max()) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("dim,N,p,q", [(3, 8, 1, 0), (3, 6, 2, 2), (2, 30, 3, 6)])
def test_reordered_mesh_action(setup, prec, dim, N, p, q):
    """The action on a randomly numbered mesh, renumbered by the Morton + first-touch
    ordering, is the same operator: y' = A'(P u) gives y = P^T y'."""
    import oracle
    from feinputs import shuffled_mesh
    fe, _, _ = setup
    m = shuffled_mesh(structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=30 + N), 31)
    perm, vnew, nnew = fe.mesh_order(dim, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    x2, c2v, c2n = fe.apply_mesh_order(m.coords, m.cell2vertex, m.cell2node, perm, vnew, nnew)
    kind = fe.ELASTICITY if dim == 3 else fe.MASS
    nc = dim if kind == fe.ELASTICITY else 1
    kw = dict(lam=1.25, mu=1.0) if kind == fe.ELASTICITY else {}
    u = uniform_field(m.n_nodes * nc, 32)
    M1 = fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    M2 = fe.Mesh(dim, p, x2, c2v, c2n, m.n_nodes)
    y1 = fe.Plan(M1, kind, q, precision=prec, **kw).apply(torch.from_numpy(u).cuda()).cpu().numpy()
    y2 = fe.Plan(M2, kind, q, precision=prec, **kw).apply(
        torch.from_numpy(fe.permute_dofs(u, nnew, nc)).cuda()).cpu().numpy()
    back = fe.unpermute_dofs(y2, nnew, nc)
    o = oracle.Oracle(dim, p, q, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    ref = o.elasticity(u, 1.25, 1.0) if kind == fe.ELASTICITY else o.mass(u)
    tol = {"fp64": 1e-12, "fp32": 5e-5, "fp16": 8 * 2.0 ** -11}[prec]
    assert np.abs(back - ref).max() <= tol * np.abs(ref).max()
    assert np.abs(y1 - ref).max() <= tol * np.abs(ref).max()
