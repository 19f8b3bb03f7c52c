"""GPU parity: the CUDA action (through the C-ABI) against the CPU oracle.

Tolerance: FP64 results must agree norm-wise, ||y - y_ref||_inf / ||y_ref||_inf
<= 1e-12 (atomic scatter order makes bitwise equality impossible; the kernels
and the oracle round differently, but both are FP64 evaluations of the same
quadrature sum, so the gap is a few hundred ulps at most).
"""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement
from precision_bounds import record

pytestmark = pytest.mark.gpu
TOL = 1e-12
# The Neo-Hookean residual at the smooth sum-of-sinusoids displacement on the
# 256^2 P4 mesh is ill-conditioned in FP64: the displacement gradient is a sum of
# nodal terms ~1e3 times larger than the result, so a half-ulp change of the
# tabulation alone moves the oracle's own output by 1.5e-12 relative
# (tests/test_oracle_conditioning.py pins this).  Parity there is 1e-11.
TOL_NH_SMOOTH = 1e-11


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_17471_gb300 as fe
    assert torch.cuda.is_available()
    return fe


def rel(a, b):
    a = a.detach().cpu().numpy() if torch.is_tensor(a) else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make(fe, dim, N, p, seed=0):
    m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)
    M = fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    return m, M


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------- small cases
MASS_CASES = [(2, 13, p) for p in range(1, 7)] + [(3, 5, p) for p in range(1, 5)]


@pytest.mark.parametrize("dim,N,p", MASS_CASES)
def test_mass_parity(fe, dim, N, p):
    m, M = make(fe, dim, N, p, seed=p)
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes, 10 + p)
    plan = fe.Plan(M, fe.MASS, q)
    assert m.n_cells > 2 * 128 and m.n_cells % 128 != 0  # several CTAs and a ragged tail
    y = plan.apply(cuda(u))
    assert rel(y, o.mass(u)) <= TOL
    assert plan.status() == 0


ELAST_CASES = [(2, 11, p) for p in range(1, 5)] + [(3, 5, 1), (3, 5, 2)]


@pytest.mark.parametrize("dim,N,p", ELAST_CASES)
def test_elasticity_parity(fe, dim, N, p):
    m, M = make(fe, dim, N, p, seed=20 + p)
    q = 2 * (p - 1)
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes * dim, 30 + p)
    plan = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0)
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL
    # the paper's constants lambda = 0, mu = 1/2
    plan2 = fe.Plan(M, fe.ELASTICITY, q, lam=0.0, mu=0.5)
    assert rel(plan2.apply(cuda(u)), o.elasticity(u, 0.0, 0.5)) <= TOL


NH_CASES = [(2, 9, p) for p in range(1, 5)] + [(3, 5, 1), (3, 5, 2)]


@pytest.mark.parametrize("dim,N,p", NH_CASES)
def test_nh_residual_jacobian_adjoint_parity(fe, dim, N, p):
    m, M = make(fe, dim, N, p, seed=40 + p)
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 50 + p)
    u = sinusoid_displacement(m, 60 + p)
    w = uniform_field(m.n_nodes * dim, 70 + p)
    res = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam)
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL
    jac = fe.Plan(M, fe.NH_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(u))
    assert rel(jac.apply(cuda(w)), o.nh_jacobian(u, w, mu, lam)) <= TOL
    jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, ojtw) <= TOL
    assert rel(dmu, odmu) <= TOL
    assert rel(dlam, odlam) <= TOL
    assert res.status() == 0 and jac.status() == 0


def test_nh_constant_coefficients(fe):
    m, M = make(fe, 2, 7, 3, seed=3)
    o = oracle.Oracle.from_mesh(m, 6)
    u = sinusoid_displacement(m, 1)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 6, mu=1.0, lam=1.25)
    ones = np.ones(m.n_cells)
    assert rel(plan.apply(cuda(u)), o.nh_residual(u, ones, 1.25 * ones)) <= TOL


# ---------------------------------------------------------------- full-size workloads
def test_full_mass_p2_2d_n64(fe):
    m, M = make(fe, 2, 64, 2, seed=20250617)
    o = oracle.Oracle.from_mesh(m, 4)
    u = uniform_field(m.n_nodes, 1)
    y = fe.Plan(M, fe.MASS, 4).apply(cuda(u))
    assert rel(y, o.mass(u, threads=8)) <= TOL
    assert abs(float(fe.Plan(M, fe.MASS, 4).apply(torch.ones(m.n_nodes, dtype=torch.float64,
                                                             device="cuda")).sum()) - 1.0) < 1e-13


def test_full_elasticity_p2_3d_n32(fe):
    m, M = make(fe, 3, 32, 2, seed=20250618)
    o = oracle.Oracle.from_mesh(m, 2)
    u = uniform_field(m.n_nodes * 3, 2)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0)
    y = plan.apply(cuda(u))
    assert rel(y, o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    assert plan.status() == 0


def test_full_nh_p4_2d_n256(fe):
    m, M = make(fe, 2, 256, 4, seed=20250619)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    w = uniform_field(m.n_nodes * 2, 5)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam)
    r = plan.apply(cuda(u))
    err = rel(r, o.nh_residual(u, mu, lam, threads=16))
    record("nh_residual", "fp64", err, "p4 2d N256 smooth field")
    assert err <= TOL_NH_SMOOTH
    jtw, dmu, dlam = plan.adjoint(cuda(u), cuda(w))
    # J^T w over the whole mesh against the oracle's Jacobian action (the two are
    # equal by the tangent's symmetry, pinned on the CPU) ...
    err = rel(jtw, o.nh_jacobian(u, w, mu, lam, threads=16))
    record("nh_adjoint_jtw", "fp64", err, "p4 2d N256 smooth field")
    assert err <= TOL
    # ... and the literal transposed-element-matrix adjoint on sampled cell ranges
    for c0, c1 in ((0, 1500), (m.n_cells // 2, m.n_cells // 2 + 1500), (m.n_cells - 1500, m.n_cells)):
        _, odmu, odlam = o.nh_adjoint(u, w, mu, lam, threads=8, cells=(c0, c1))
        # dmu, dlambda integrate F - F^{-T} and ln(det F) F^{-T}: smooth-field conditioned
        e_mu, e_lam = rel(dmu[c0:c1], odmu[c0:c1]), rel(dlam[c0:c1], odlam[c0:c1])
        record("nh_adjoint_dmu", "fp64", e_mu, f"p4 2d N256 cells {c0}-{c1}")
        record("nh_adjoint_dlam", "fp64", e_lam, f"p4 2d N256 cells {c0}-{c1}")
        assert e_mu <= TOL_NH_SMOOTH
        assert e_lam <= TOL_NH_SMOOTH
    assert plan.status() == 0


# ---------------------------------------------------------------- edge cases
def test_empty_mesh_zeroes_output(fe):
    m = structured_mesh(2, 2, 2)
    M = fe.Mesh(2, 2, m.coords, m.cell2vertex[:0], m.cell2node[:0], m.n_nodes)
    y = torch.full((m.n_nodes,), 7.0, dtype=torch.float64, device="cuda")
    fe.Plan(M, fe.MASS, 4).apply(torch.ones_like(y), y)
    assert float(y.abs().max()) == 0.0


def test_single_cell(fe):
    m = structured_mesh(2, 1, 3, seed=0)
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex[:1], m.cell2node[:1], m.n_nodes)
    u = uniform_field(m.n_nodes * 2, 9)
    plan = fe.Plan(M, fe.ELASTICITY, 4, lam=1.25, mu=1.0)
    o = oracle.Oracle(2, 3, 4, m.coords, m.cell2vertex[:1], m.cell2node[:1], m.n_nodes)
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL


def test_accumulate_flag(fe):
    m, M = make(fe, 2, 8, 2)
    o = oracle.Oracle.from_mesh(m, 4)
    u = uniform_field(m.n_nodes, 1)
    y0 = uniform_field(m.n_nodes, 2)
    y = cuda(y0.copy())
    fe.Plan(M, fe.MASS, 4, accumulate=True).apply(cuda(u), y)
    assert rel(y, y0 + o.mass(u)) <= TOL


def test_nondefault_stream_and_host_path(fe):
    m, M = make(fe, 2, 16, 4)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 1)
    u = sinusoid_displacement(m, 2)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y = plan.apply(cuda(u))
    s.synchronize()
    ref = o.nh_residual(u, mu, lam)
    assert rel(y, ref) <= TOL
    yh = plan.apply_host(torch.from_numpy(u).pin_memory())
    assert not yh.is_cuda and rel(yh.numpy(), ref) <= TOL


def test_out_of_range_index_sets_status(fe):
    m = structured_mesh(2, 6, 2, jitter=0.1, seed=1)
    c2n = m.cell2node.copy()
    c2n[17, 3] = m.n_nodes + 5
    M = fe.Mesh(2, 2, m.coords, m.cell2vertex, c2n, m.n_nodes)
    plan = fe.Plan(M, fe.MASS, 4)
    plan.apply(torch.ones(m.n_nodes, dtype=torch.float64, device="cuda"))
    assert plan.status() == 5  # FE_ERR_INDEX, no fault
    c2v = m.cell2vertex.copy()
    c2v[3, 1] = -1
    M2 = fe.Mesh(2, 2, m.coords, c2v, m.cell2node, m.n_nodes)
    plan2 = fe.Plan(M2, fe.MASS, 4)
    plan2.apply(torch.ones(m.n_nodes, dtype=torch.float64, device="cuda"))
    assert plan2.status() == 5
    assert plan2.status() == 0  # reading clears it


def test_degenerate_cell_sets_status(fe):
    m = structured_mesh(2, 4, 1)
    coords = m.coords.copy()
    coords[m.cell2vertex[5, 2]] = coords[m.cell2vertex[5, 0]]
    M = fe.Mesh(2, 1, coords, m.cell2vertex, m.cell2node, m.n_nodes)
    plan = fe.Plan(M, fe.MASS, 2)
    plan.apply(torch.ones(m.n_nodes, dtype=torch.float64, device="cuda"))
    assert plan.status() == 4  # FE_ERR_BAD_MESH


def test_inverted_deformation_sets_status_and_nan_propagates(fe):
    m, M = make(fe, 2, 4, 2)
    mu, lam = lame_fields(m.n_cells, 1)
    # u = (-3x, 0): F = diag(-2, 1), det F = -2 < 0 everywhere
    u = np.zeros((m.n_nodes, 2))
    u[:, 0] = -3.0 * m.node_lattice[:, 0] / (2 * 4)
    u = u.reshape(-1)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 4, mu_cell=mu, lam_cell=lam)
    y = plan.apply(cuda(u))
    assert plan.status() == 8  # FE_ERR_NONFINITE
    assert torch.isnan(y).any()
    un = uniform_field(m.n_nodes * 2, 3) * 0.01
    un[4] = np.nan
    y = plan.apply(cuda(un))
    assert torch.isnan(y).any()


def test_invalid_arguments_rejected(fe):
    from paper_2506_17471_gb300 import FeError
    m, M = make(fe, 2, 4, 2)
    plan = fe.Plan(M, fe.MASS, 4)
    with pytest.raises(ValueError):
        plan.apply(torch.ones(3, dtype=torch.float64, device="cuda"))
    u = torch.ones(m.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(FeError):
        plan.adjoint(u, u)  # only the Neo-Hookean residual has an adjoint
    with pytest.raises(FeError):
        fe.Plan(M, 7, 4)


# ---------------------------------------------------------------- autograd
def test_autograd_function_matches_oracle_and_fd(fe):
    m, M = make(fe, 2, 6, 4, seed=9)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 11)
    u = sinusoid_displacement(m, 12)
    w = uniform_field(m.n_nodes * 2, 13)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam)
    ut = cuda(u).requires_grad_(True)
    mut = cuda(mu).requires_grad_(True)
    lamt = cuda(lam).requires_grad_(True)
    r = fe.NeoHookeanResidual.apply(ut, mut, lamt, plan)
    (r * cuda(w)).sum().backward()
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(ut.grad, ojtw) <= TOL
    assert rel(mut.grad, odmu) <= TOL
    assert rel(lamt.grad, odlam) <= TOL
    # FP64 central differences of w . r along a random direction (h = 1e-6)
    d = uniform_field(m.n_nodes * 2, 14)
    h = 1e-6
    with torch.no_grad():
        rp = fe.NeoHookeanResidual.apply(cuda(u + h * d), mut, lamt, plan)
        rm = fe.NeoHookeanResidual.apply(cuda(u - h * d), mut, lamt, plan)
        fd = float(((rp - rm) * cuda(w)).sum()) / (2 * h)
    an = float((ut.grad * cuda(d)).sum())
    assert abs(fd - an) <= 1e-7 * abs(an)


def test_autograd_second_forward_does_not_change_first_gradients(fe):
    """Two forwards on one plan with different Lame fields, then backpropagation
    through the first: its gradients use the first call's fields."""
    m, M = make(fe, 2, 6, 4, seed=19)
    o = oracle.Oracle.from_mesh(m, 8)
    mu1, lam1 = lame_fields(m.n_cells, 21)
    mu2, lam2 = lame_fields(m.n_cells, 22)
    u = sinusoid_displacement(m, 23)
    w = uniform_field(m.n_nodes * 2, 24)
    plan = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu1, lam_cell=lam1)
    ut = cuda(u).requires_grad_(True)
    mut = cuda(mu1).requires_grad_(True)
    lamt = cuda(lam1).requires_grad_(True)
    r1 = fe.NeoHookeanResidual.apply(ut, mut, lamt, plan)
    r2 = fe.NeoHookeanResidual.apply(cuda(u), cuda(mu2), cuda(lam2), plan)
    assert rel(r2, o.nh_residual(u, mu2, lam2)) <= TOL
    (r1 * cuda(w)).sum().backward()
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu1, lam1)
    assert rel(ut.grad, ojtw) <= TOL
    assert rel(mut.grad, odmu) <= TOL
    assert rel(lamt.grad, odlam) <= TOL


def test_plans_of_one_kernel_keep_their_shared_memory(fe):
    """A later plan of the same kernel with a smaller table must not break an
    earlier plan that needs more dynamic shared memory."""
    m, M = make(fe, 2, 6, 4, seed=3)
    o_big = oracle.Oracle.from_mesh(m, 30)
    big = fe.Plan(M, fe.MASS, 30)      # 256-point rule: ~95 KB table
    small = fe.Plan(M, fe.MASS, 2)     # 4-point rule: ~1.6 KB table
    u = uniform_field(m.n_nodes, 1)
    assert rel(big.apply(cuda(u)), o_big.mass(u)) <= TOL
    assert rel(small.apply(cuda(u)), oracle.Oracle.from_mesh(m, 2).mass(u)) <= TOL
    c = structured_mesh(3, 3, 4, jitter=0.15, seed=2)
    C = fe.Mesh(3, 4, c.coords, c.cell2vertex, c.cell2node, c.n_nodes)
    wide = fe.Plan(C, fe.ELASTICITY, 6, lam=1.25, mu=1.0, tile_cells=5)
    narrow = fe.Plan(C, fe.ELASTICITY, 6, lam=1.25, mu=1.0, tile_cells=1)
    v = uniform_field(c.n_nodes * 3, 2)
    ref = oracle.Oracle.from_mesh(c, 6).elasticity(v, 1.25, 1.0)
    assert rel(wide.apply(cuda(v)), ref) <= TOL and rel(narrow.apply(cuda(v)), ref) <= TOL


# ---------------------------------------------------------------- fully symmetric rules
@pytest.mark.parametrize("dim,N,p,form,q", [(2, 13, 2, "mass", 4), (2, 9, 3, "mass", 6),
                                            (3, 5, 2, "elasticity", 2), (2, 11, 4, "elasticity", 6),
                                            (3, 4, 3, "mass", 5), (2, 9, 4, "nh", 8), (3, 5, 2, "nh", 4)])
def test_symmetric_rules_parity(fe, dim, N, p, form, q):
    m, M = make(fe, dim, N, p, seed=500 + p)
    o = oracle.Oracle.from_mesh(m, q, "symmetric")
    if form == "mass":
        u = uniform_field(m.n_nodes, 1)
        plan = fe.Plan(M, fe.MASS, q, quad_scheme="symmetric")
        assert plan.info.nq == o.nq
        assert rel(plan.apply(cuda(u)), o.mass(u)) <= TOL
    elif form == "elasticity":
        u = uniform_field(m.n_nodes * dim, 2)
        plan = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0, quad_scheme="symmetric")
        assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL
    else:
        mu, lam = lame_fields(m.n_cells, 3)
        u = sinusoid_displacement(m, 4)
        w = uniform_field(m.n_nodes * dim, 5)
        res = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam, quad_scheme="symmetric")
        assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL
        jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
        ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
        assert rel(jtw, ojtw) <= TOL and rel(dmu, odmu) <= TOL
        coop = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam, quad_scheme="symmetric",
                       cooperative=True)
        assert rel(coop.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL


def test_full_elasticity_p2_3d_n32_symmetric_rule(fe):
    """The benchmark workload with the 4-point degree-2 rule."""
    m, M = make(fe, 3, 32, 2, seed=20250618)
    o = oracle.Oracle.from_mesh(m, 2, "symmetric")
    assert o.nq == 4
    u = uniform_field(m.n_nodes * 3, 2)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0, quad_scheme="symmetric")
    assert plan.info.nq == 4
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL
    assert plan.status() == 0


@pytest.mark.parametrize("block", [32, 64, 96, 128])
def test_tpc_block_sizes(fe, block):
    """Threads per block of the thread-per-cell kernel (the paper's work-group
    size): every size gives the same action; other sizes are refused."""
    m = structured_mesh(2, 20, 3, jitter=0.2, seed=61)
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    o = oracle.Oracle.from_mesh(m, 4)
    u = uniform_field(m.n_nodes * 2, 62)
    plan = fe.Plan(M, fe.ELASTICITY, 4, lam=1.25, mu=1.0, tile_cells=block)
    assert plan.info.kernel == 0 and plan.info.threads_per_block == block
    y = plan.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert np.abs(y - o.elasticity(u, 1.25, 1.0)).max() <= 1e-12 * np.abs(y).max()
    assert plan.status() == 0
    with pytest.raises(Exception):
        fe.Plan(M, fe.ELASTICITY, 4, lam=1.25, mu=1.0, tile_cells=48)


def test_bounded_wait_times_out_and_context_survives(fe):
    """Failure detection without a GPU fault: a kernel waits on an mbarrier that
    nothing ever completes; the kernels' bounded wait gives up, FE_ERR_TIMEOUT
    reaches the host through the status word, and the context keeps working."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert N.lib.fe_selftest_bounded_wait(ctypes.c_void_p(st.data_ptr()), 4096, None) == N.FE_OK
    torch.cuda.synchronize()
    assert int(st.item()) == N.FE_ERR_TIMEOUT
    assert N.lib.fe_selftest_bounded_wait(None, 10, None) == N.FE_ERR_INVALID_ARG
    assert N.lib.fe_selftest_bounded_wait(ctypes.c_void_p(st.data_ptr()), 0, None) == N.FE_ERR_INVALID_ARG
    m = structured_mesh(2, 8, 2, jitter=0.2, seed=3)
    M = fe.Mesh(2, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    u = uniform_field(m.n_nodes, 4)
    plan = fe.Plan(M, fe.MASS, 4)
    y = plan.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel(y, oracle.Oracle.from_mesh(m, 4).mass(u)) <= TOL and plan.status() == 0
