"""GPU parity of the Laplacian, Helmholtz and St. Venant-Kirchhoff actions
(Appendix A) against the FP64 oracle: thread-per-cell and cells-per-CTA kernels,
FP64 (tolerance 1e-12 norm-wise) and FP32 contractions (5e-5, the FP32 bound of
tests/test_mixed_gpu.py), several tiles with ragged tails, the paper's Helmholtz
P4 rows, edge cases."""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL32 = 5e-5


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


def make(fe, dim, N, p, seed):
    m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)
    return m, fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)


def run(fe, kind, dim, N, p, q, prec="fp64", coop=False, scheme="conical", seed=0):
    m, M = make(fe, dim, N, p, 700 + 10 * dim + p + seed)
    o = oracle.Oracle.from_mesh(m, q, scheme=scheme)
    name = fe.FORM_NAMES[kind]
    if kind in (fe.LAPLACE, fe.HELMHOLTZ):
        u = uniform_field(m.n_nodes, 3 + p)
        plan = fe.Plan(M, kind, q, precision=prec, cooperative=coop, quad_scheme=scheme)
        ref = getattr(o, name)(u)
        y = plan.apply(cuda(u))
    else:
        mu, lam = lame_fields(m.n_cells, 4 + p)
        ul = sinusoid_displacement(m, 5 + p)
        if kind == fe.SVK_RESIDUAL:
            plan = fe.Plan(M, kind, q, mu_cell=mu, lam_cell=lam, precision=prec, cooperative=coop,
                           quad_scheme=scheme)
            ref = o.svk_residual(ul, mu, lam)
            y = plan.apply(cuda(ul))
        else:
            du = uniform_field(m.n_nodes * dim, 6 + p)
            plan = fe.Plan(M, kind, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision=prec,
                           cooperative=coop, quad_scheme=scheme)
            ref = o.svk_jacobian(ul, du, mu, lam)
            y = plan.apply(cuda(du))
    err = rel(y, ref)
    assert plan.status() == 0
    return err, plan, m


CASES = [(2, 13, 1, 0), (2, 13, 2, 2), (2, 11, 3, 4), (2, 9, 4, 6), (3, 5, 1, 0), (3, 5, 2, 2), (3, 5, 3, 4)]


@pytest.mark.parametrize("coop", [False, True])
@pytest.mark.parametrize("dim,N,p,q", CASES)
def test_laplace_fp64(fe, dim, N, p, q, coop):
    err, plan, m = run(fe, fe.LAPLACE, dim, N, p, q, coop=coop)
    assert m.n_cells % 128 != 0 and err <= TOL, err


@pytest.mark.parametrize("coop", [False, True])
@pytest.mark.parametrize("dim,N,p,q", [(2, 13, 1, 2), (2, 13, 2, 4), (2, 11, 4, 8), (3, 5, 1, 2),
                                       (3, 5, 2, 4), (3, 4, 4, 8)])
def test_helmholtz_fp64(fe, dim, N, p, q, coop):
    err, plan, m = run(fe, fe.HELMHOLTZ, dim, N, p, q, coop=coop)
    assert err <= TOL, err


@pytest.mark.parametrize("kind", ["svk_residual", "svk_jacobian"])
@pytest.mark.parametrize("coop", [False, True])
@pytest.mark.parametrize("dim,N,p,q", [(2, 13, 1, 2), (2, 11, 2, 4), (2, 9, 3, 6), (2, 7, 4, 8),
                                       (3, 5, 1, 2), (3, 4, 2, 4)])
def test_svk_fp64(fe, kind, dim, N, p, q, coop):
    k = fe.SVK_RESIDUAL if kind == "svk_residual" else fe.SVK_JACOBIAN
    err, plan, m = run(fe, k, dim, N, p, q, coop=coop)
    assert err <= TOL, err


@pytest.mark.parametrize("kind,dim,N,p,q,coop", [("laplace", 2, 13, 2, 2, False), ("laplace", 2, 9, 4, 6, False),
                                                 ("laplace", 3, 5, 2, 2, True), ("helmholtz", 2, 11, 4, 8, False),
                                                 ("helmholtz", 3, 4, 4, 8, True),
                                                 ("svk_residual", 2, 11, 2, 4, False),
                                                 ("svk_jacobian", 2, 11, 2, 4, False),
                                                 ("svk_jacobian", 3, 4, 2, 4, True)])
def test_forms_fp32(fe, kind, dim, N, p, q, coop):
    err, plan, m = run(fe, getattr(fe, kind.upper()), dim, N, p, q, prec="fp32", coop=coop)
    assert 1e-12 < err <= TOL32, err


@pytest.mark.parametrize("dim,N,scheme", [(2, 64, "symmetric"), (3, 8, "conical")])
def test_helmholtz_p4_paper_rows(fe, dim, N, scheme):
    """Table "action_param_space": Helmholtz P4 in 2D (16-point degree-8 rule) and 3D."""
    err, plan, m = run(fe, fe.HELMHOLTZ, dim, N, 4, 8, scheme=scheme)
    assert plan.info.n_loc == (15 if dim == 2 else 35)
    assert err <= TOL, err


def test_forms_edge_cases(fe):
    m, M = make(fe, 2, 4, 2, 77)
    M0 = fe.Mesh(2, 2, m.coords, m.cell2vertex[:0], m.cell2node[:0], m.n_nodes)
    for kind in (fe.LAPLACE, fe.HELMHOLTZ):
        y = fe.Plan(M0, kind, 2).apply(cuda(np.ones(m.n_nodes)))
        assert float(y.abs().max()) == 0.0
    # Jacobian kinds need a linearisation point
    with pytest.raises(Exception):
        fe.Plan(M, fe.SVK_JACOBIAN, 2, mu=1.0, lam=1.0)
    # accumulate
    o = oracle.Oracle.from_mesh(m, 2)
    u, y0 = uniform_field(m.n_nodes, 1), uniform_field(m.n_nodes, 2)
    y = fe.Plan(M, fe.LAPLACE, 2, accumulate=True).apply(cuda(u), cuda(y0.copy()))
    assert rel(y, y0 + o.laplace(u)) <= TOL


def test_elasticity_p1_3d_paper_size(fe):
    """Elasticity P1 on ~1e6 tetrahedra (the paper's H200 3D problem size, and the
    case of its low-order traffic analysis): every output against the oracle."""
    m, M = make(fe, 3, 55, 1, 55)
    assert m.n_cells == 998250
    o = oracle.Oracle.from_mesh(m, 0)
    u = uniform_field(m.n_nodes * 3, 56)
    plan = fe.Plan(M, fe.ELASTICITY, 0, lam=1.25, mu=1.0)
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    assert plan.status() == 0
