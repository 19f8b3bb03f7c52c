"""GPU parity of the cooperative (cells-per-CTA) kernel against the FP64 oracle.

Small meshes cover several CTA batches and a ragged last batch, both at degrees
that also have a thread-per-cell kernel (forced with ``cooperative=True``) and
at the high degrees only this kernel serves.  The hp-sweep workloads (about 4M
DoFs) are compared in full; at about 16M DoFs the oracle recomputes sampled
output DoFs exactly, from the cells that contain them.
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
TOL32 = 5e-5
# Neo-Hookean tangent linearised at the smooth sinusoid field on the fine P6 mesh:
# FP64 conditioning (tests/test_oracle_conditioning.py) puts independent
# evaluations ~1e-12 apart; parity there is 1e-11, and a small random
# linearisation point (well conditioned) is held to 1e-12.
TOL_NH_SMOOTH = 1e-11


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


CASES = [(2, 9, 2), (2, 7, 4), (2, 5, 6), (2, 4, 8), (3, 4, 2), (3, 3, 3), (3, 2, 4)]


@pytest.mark.parametrize("dim,N,p", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coop_linear_forms(fe, dim, N, p, prec):
    m, M = make(fe, dim, N, p, 200 + p)
    tol = TOL if prec == "fp64" else TOL32
    o = oracle.Oracle.from_mesh(m, 2 * p)
    u = uniform_field(m.n_nodes, 1)
    plan = fe.Plan(M, fe.MASS, 2 * p, precision=prec, cooperative=True)
    assert plan.info.kernel == 1
    assert rel(plan.apply(cuda(u)), o.mass(u)) <= tol
    q = 2 * (p - 1)
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes * dim, 2)
    plan = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0, precision=prec, cooperative=True)
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= tol
    assert plan.status() == 0


@pytest.mark.parametrize("dim,N,p", CASES)
def test_coop_neo_hookean(fe, dim, N, p):
    m, M = make(fe, dim, N, p, 300 + p)
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    w = uniform_field(m.n_nodes * dim, 5)
    res = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam, cooperative=True)
    assert res.info.kernel == 1
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL
    jac = fe.Plan(M, fe.NH_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(u), cooperative=True)
    assert rel(jac.apply(cuda(w)), o.nh_jacobian(u, w, mu, lam)) <= TOL
    jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, ojtw) <= TOL
    assert rel(dmu, odmu) <= TOL and rel(dlam, odlam) <= TOL
    assert res.status() == 0 and jac.status() == 0


def test_high_degree_selects_cooperative_kernel(fe):
    m, M = make(fe, 2, 3, 6, 1)
    mu, lam = lame_fields(m.n_cells, 1)
    u = sinusoid_displacement(m, 2)
    jac = fe.Plan(M, fe.NH_JACOBIAN, 12, mu_cell=mu, lam_cell=lam, u_lin=cuda(u))
    assert jac.info.kernel == 1
    m3, M3 = make(fe, 3, 2, 4, 1)
    assert fe.Plan(M3, fe.ELASTICITY, 6, lam=1.25, mu=1.0).info.kernel == 1
    assert fe.Plan(M3, fe.MASS, 8).info.kernel == 0   # thread-per-cell exists for mass P4 3D


def sampled_oracle(m, q, nodes, fn):
    """Oracle output at the given nodes, from exactly the cells that contain them."""
    cells = np.unique(np.nonzero(np.isin(m.cell2node, nodes))[0])
    o = oracle.Oracle(m.dim, m.degree, q, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes)
    return fn(o, cells)


HP = [  # (name, dim, degree, N, q) of the hp sweep at ~4M and ~16M DoFs
    ("nh_jacobian_p6_2d", 2, 6, 236, 12), ("nh_jacobian_p6_2d", 2, 6, 471, 12),
    ("elasticity_p4_3d", 3, 4, 27, 6), ("elasticity_p4_3d", 3, 4, 43, 6),
    ("mass_p3_2d", 2, 3, 667, 6), ("mass_p3_2d", 2, 3, 1333, 6),
]


@pytest.mark.parametrize("name,dim,p,N,q", HP)
def test_hp_sweep_full_size(fe, name, dim, p, N, q):
    m, M = make(fe, dim, N, p, 20250620 + N)
    big = N in (471, 43, 1333)
    if name == "mass_p3_2d":
        u = uniform_field(m.n_nodes, 1)
        y = fe.Plan(M, fe.MASS, q).apply(cuda(u)).cpu().numpy()
        fn = lambda o, cells: o.mass(u, threads=16)
        ncomp = 1
    elif name == "elasticity_p4_3d":
        u = uniform_field(m.n_nodes * 3, 1)
        y = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0).apply(cuda(u)).cpu().numpy()
        fn = lambda o, cells: o.elasticity(u, 1.25, 1.0, threads=16)
        ncomp = 3
    else:
        mu, lam = lame_fields(m.n_cells, 2)
        ul = sinusoid_displacement(m, 3)
        du = uniform_field(m.n_nodes * 2, 4)
        plan = fe.Plan(M, fe.NH_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul))
        y = plan.apply(cuda(du)).cpu().numpy()
        fn = lambda o, cells: o.nh_jacobian(ul, du, mu[cells] if len(cells) < m.n_cells else mu,
                                            lam[cells] if len(cells) < m.n_cells else lam, threads=16)
        ncomp = 2
    tol = TOL_NH_SMOOTH if name == "nh_jacobian_p6_2d" else TOL
    if not big:
        o = oracle.Oracle.from_mesh(m, q)
        ref = fn(o, np.arange(m.n_cells))
        err = rel(y, ref)
        record(name, "fp64", err, f"N{N} full size")
        assert err <= tol
        if name == "nh_jacobian_p6_2d":
            # well-conditioned linearisation point: random, small enough for det F > 0
            ur = uniform_field(m.n_nodes * 2, 5) * (0.004 / (p * N))
            plan.set_linearisation(cuda(ur))
            yr = plan.apply(cuda(du)).cpu().numpy()
            assert rel(yr, o.nh_jacobian(ur, du, mu, lam, threads=16)) <= TOL
    else:
        rng = np.random.default_rng(N)
        nodes = rng.choice(m.n_nodes, size=64, replace=False)
        ref = sampled_oracle(m, q, nodes, fn)
        idx = (nodes[:, None] * ncomp + np.arange(ncomp)[None, :]).reshape(-1)
        err = np.abs(y[idx] - ref[idx]).max() / np.abs(y).max()
        record(name, "fp64", err, f"N{N} sampled DoFs")
        assert err <= tol


@pytest.mark.parametrize("dim,N,p", [(2, 5, 6), (3, 3, 3), (3, 2, 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coop_tables_in_global_memory(fe, dim, N, p, prec):
    """Cells-per-CTA kernel with the tabulation kept in global memory (two
    coalesced layouts) instead of shared memory."""
    m, M = make(fe, dim, N, p, 400 + p)
    tol = TOL if prec == "fp64" else TOL32
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    w = uniform_field(m.n_nodes * dim, 5)
    res = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam, precision=prec, cooperative=True,
                  tables_global=True)
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= tol
    jtw, dmu, _ = res.adjoint(cuda(u), cuda(w))
    ojtw, odmu, _ = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, ojtw) <= tol
    s = uniform_field(m.n_nodes, 6)
    mp = fe.Plan(M, fe.MASS, q, precision=prec, cooperative=True, tables_global=True, tile_cells=7)
    assert rel(mp.apply(cuda(s)), o.mass(s)) <= tol
    assert res.status() == 0 and mp.status() == 0


@pytest.mark.parametrize("prec", ["fp32"])
def test_hp_mass_p3_reduced_precision_full_size(fe, prec):
    """hp-sweep size mass P3 (4,008,004 DoFs) with FP32 contractions: every DoF
    within the FP32 bound of the FP64 oracle."""
    m, M = make(fe, 2, 667, 3, 20250620 + 667)
    u = uniform_field(m.n_nodes, 1)
    plan = fe.Plan(M, fe.MASS, 6, precision=prec)
    y = plan.apply(cuda(u)).cpu().numpy()
    ref = oracle.Oracle.from_mesh(m, 6).mass(u, threads=16)
    assert rel(y, ref) <= TOL32
    assert plan.status() == 0


@pytest.mark.parametrize("N", [3, 4])
def test_coop_elasticity_p4_3d_symmetric_rule(fe, N):
    """Elasticity P4 tets with the 24-point fully symmetric degree-6 rule on the
    cells-per-CTA kernel (the benchmark's configuration): several CTA batches and
    a ragged last batch (162 and 384 cells)."""
    m, M = make(fe, 3, N, 4, 500 + N)
    o = oracle.Oracle.from_mesh(m, 6, "symmetric")
    assert o.nq == 24
    u = uniform_field(m.n_nodes * 3, 7)
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, quad_scheme="symmetric")
    assert plan.info.kernel == 1 and plan.info.nq == 24
    assert rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL
    # a degree-6-exact rule integrates the degree-6 integrand exactly on affine
    # cells, so the 64-point conical-product rule gives the same action
    conical = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0)
    assert conical.info.nq == 64
    assert rel(conical.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)) <= TOL
    assert plan.status() == 0 and conical.status() == 0


@pytest.mark.parametrize("name", ["elasticity_p4_3d_n27", "elasticity_p4_3d_n43"])
def test_benchmark_workload_full_size(fe, name):
    """The benchmark's workloads exactly as it builds them (same generators, same
    plan options, so the same launch configuration): at ~4M DoFs every DoF against
    the oracle; at ~16M DoFs sampled output DoFs recomputed by the oracle from the
    cells that contain them."""
    from feinputs import workloads
    wl = {w.name: w for w in (workloads.ELASTICITY_P4_3D_N27, workloads.ELASTICITY_P4_3D_N43)}[name]
    m = wl.mesh()
    M = fe.Mesh(3, wl.degree, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    u = wl.field(m)
    plan = fe.Plan(M, fe.ELASTICITY, wl.quad_degree, lam=wl.lam, mu=wl.mu, quad_scheme=wl.quad_scheme)
    assert plan.info.kernel == 1
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == 0
    if wl.N <= 27:
        ref = oracle.Oracle.from_mesh(m, wl.quad_degree, wl.quad_scheme).elasticity(u, wl.lam, wl.mu, threads=16)
        assert rel(y, ref) <= TOL
    else:
        rng = np.random.default_rng(wl.N)
        nodes = rng.choice(m.n_nodes, size=64, replace=False)
        cells = np.unique(np.nonzero(np.isin(m.cell2node, nodes))[0])
        o = oracle.Oracle(3, wl.degree, wl.quad_degree, m.coords, m.cell2vertex[cells], m.cell2node[cells],
                          m.n_nodes, wl.quad_scheme)
        ref = o.elasticity(u, wl.lam, wl.mu, threads=16)
        idx = (nodes[:, None] * 3 + np.arange(3)[None, :]).reshape(-1)
        assert np.abs(y[idx] - ref[idx]).max() <= TOL * np.abs(y).max()
