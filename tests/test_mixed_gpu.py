"""GPU parity of the FP32-contraction (mixed-precision) kernels against the FP64 oracle.

Stated bound: tables, DoFs and accumulators are IEEE single (unit roundoff
u = 2^-24 = 6.0e-8); each evaluation contraction has at most d*n_loc <= 105
terms and each quadrature contraction at most Q(1+d) <= 256 terms, so the
forward error of each contraction is at most gamma_256 = 256u/(1-256u) = 1.5e-5
of the sum of the absolute terms.  For the random inputs below the absolute
terms exceed the result by a small factor, and the parity tolerance is
TOL32 = 5e-5 (norm-wise, relative to ||y_ref||_inf).  Geometry, the
Neo-Hookean kinematics/stress/log and the scatter are FP64 and add nothing at
this level.  The hyperelastic forms evaluate gradients of a smooth displacement
that are ~1e3 times smaller than the nodal values (see
tests/test_oracle_conditioning.py); the kernels gather those DoFs relative to
each cell's first node in FP64 before rounding to single, so the rounding acts
on the cell-local variation only and the same TOL32 holds for them.
"""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu
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


@pytest.mark.parametrize("dim,N,p", [(2, 13, 1), (2, 13, 2), (2, 13, 3), (2, 9, 6), (3, 5, 2), (3, 4, 4)])
def test_mass_fp32(fe, dim, N, p):
    m, M = make(fe, dim, N, p, 100 + p)
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes, 1)
    y = fe.Plan(M, fe.MASS, q, precision="fp32").apply(cuda(u))
    err = rel(y, o.mass(u))
    assert err <= TOL32 and err > 1e-12   # really computed in single


@pytest.mark.parametrize("dim,N,p", [(2, 11, 2), (2, 11, 4), (3, 5, 1), (3, 5, 2)])
def test_elasticity_fp32(fe, dim, N, p):
    m, M = make(fe, dim, N, p, 110 + p)
    q = 2 * (p - 1)
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes * dim, 2)
    y = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0, precision="fp32").apply(cuda(u))
    assert rel(y, o.elasticity(u, 1.25, 1.0)) <= TOL32


@pytest.mark.parametrize("dim,N,p", [(2, 9, 2), (2, 9, 4), (3, 5, 2)])
def test_nh_fp32(fe, dim, N, p):
    m, M = make(fe, dim, N, p, 120 + p)
    q = 2 * p
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    w = uniform_field(m.n_nodes * dim, 5)
    res = fe.Plan(M, fe.NH_RESIDUAL, q, mu_cell=mu, lam_cell=lam, precision="fp32")
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam)) <= TOL32
    jac = fe.Plan(M, fe.NH_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(u), precision="fp32")
    assert rel(jac.apply(cuda(w)), o.nh_jacobian(u, w, mu, lam)) <= TOL32
    jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
    ojtw, odmu, odlam = o.nh_adjoint(u, w, mu, lam)
    assert rel(jtw, ojtw) <= TOL32
    assert rel(dmu, odmu) <= TOL32 and rel(dlam, odlam) <= TOL32


def test_full_elasticity_p2_3d_fp32(fe):
    m, M = make(fe, 3, 32, 2, 20250618)
    o = oracle.Oracle.from_mesh(m, 2)
    u = uniform_field(m.n_nodes * 3, 2)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0, precision="fp32")
    y = plan.apply(cuda(u))
    assert rel(y, o.elasticity(u, 1.25, 1.0, threads=16)) <= TOL32
    assert plan.status() == 0


def test_bit_conversions_match_hardware(fe):
    """The mixed kernels convert binary64 <-> binary32 with branch-free integer bit
    operations (round to nearest even, values below 2^-126 flushed to signed
    zero); they must agree bit for bit with CUDA's conversion with that flush."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    rng = np.random.default_rng(0)
    vals = [rng.standard_normal(200_000) * 10.0 ** rng.integers(-45, 45, 200_000),
            rng.uniform(-1, 1, 100_000),
            np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-310, -1e-320, 3.4028234663852886e38,
                      3.4028235677973366e38, 3.402823669209385e38, 1.1754943508222875e-38,
                      1.1754942106924411e-38, 1.401298464324817e-45, 7e-46, 1e300, -1e300])]
    f = rng.standard_normal(100_000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    vals.append((f.astype(np.float64) + nxt.astype(np.float64)) / 2)     # exact ties
    x = torch.from_numpy(np.concatenate(vals)).cuda()
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc = N.lib.fe_selftest_conversions(ctypes.c_void_p(x.data_ptr()), x.numel(),
                                       ctypes.c_void_p(count.data_ptr()), None)
    assert rc == 0
    assert count.tolist() == [0, 0]


def test_full_nh_p4_2d_fp32_smooth_field(fe):
    """The ill-conditioned case at full size (256^2 x 2 P4 triangles, the smooth
    sinusoid displacement): FP32 contractions of DoFs gathered relative to each
    cell's first node keep the residual, the adjoint and the Jacobian action
    within TOL32 of the FP64 oracle (rounding the absolute DoFs to single lost
    ~1e-3)."""
    m, M = make(fe, 2, 256, 4, 20250619)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    w = uniform_field(m.n_nodes * 2, 5)
    res = fe.Plan(M, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam, precision="fp32")
    assert rel(res.apply(cuda(u)), o.nh_residual(u, mu, lam, threads=16)) <= TOL32
    jtw, dmu, dlam = res.adjoint(cuda(u), cuda(w))
    assert rel(jtw, o.nh_jacobian(u, w, mu, lam, threads=16)) <= TOL32
    _, odmu, odlam = o.nh_adjoint(u, w, mu, lam, threads=8, cells=(0, 2000))
    assert rel(dmu[:2000], odmu[:2000]) <= TOL32 and rel(dlam[:2000], odlam[:2000]) <= TOL32
    assert res.status() == 0


@pytest.mark.parametrize("block", [32, 96, 128])
@pytest.mark.parametrize("shuffled", [False, True])
def test_fp32_block_sizes_and_numberings(fe, block, shuffled):
    """FP32 thread-per-cell kernels at several block sizes, with a ragged last
    block, on the structured numbering and on a random one: mass, Laplacian,
    Helmholtz and elasticity."""
    from feinputs import shuffled_mesh
    m = structured_mesh(3, 5, 2, jitter=0.15, seed=91)
    if shuffled:
        m = shuffled_mesh(m, 92)
    M = fe.Mesh(3, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    assert m.n_cells % block != 0
    o = oracle.Oracle.from_mesh(m, 4)
    s = uniform_field(m.n_nodes, 93)
    v = uniform_field(m.n_nodes * 3, 94)
    for kind, ref, x in ((fe.MASS, o.mass, s), (fe.LAPLACE, o.laplace, s), (fe.HELMHOLTZ, o.helmholtz, s)):
        plan = fe.Plan(M, kind, 4, precision="fp32", tile_cells=block)
        assert rel(plan.apply(cuda(x)), ref(x)) <= TOL32
        assert plan.status() == 0
    plan = fe.Plan(M, fe.ELASTICITY, 4, lam=1.25, mu=1.0, precision="fp32", tile_cells=block)
    y = torch.full((m.n_nodes * 3,), 7.0, dtype=torch.float64, device="cuda")
    plan.apply(cuda(v), y)
    assert rel(y, o.elasticity(v, 1.25, 1.0)) <= TOL32
    assert plan.status() == 0


@pytest.mark.parametrize("shuffled", [False, True])
def test_fp32_mass_scatter_aggregation_full_size(fe, shuffled):
    """Mass P3 on 2 x 1333^2 triangles (16,000,000 DoFs, y = 128 MB, larger than L2):
    on the structured numbering the FP32 plan sums each 128-cell tile's updates per
    node in shared memory before the scatter; on a random numbering (no shared
    nodes within a tile) it scatters directly.  Sampled DoFs against the oracle,
    recomputed from the cells that contain them, and both against the FP64 plan."""
    from feinputs import shuffled_mesh
    m = structured_mesh(2, 1333, 3, jitter=0.2, seed=20250620 + 1333)
    if shuffled:
        m = shuffled_mesh(m, 95)
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    u = uniform_field(m.n_nodes, 96)
    plan = fe.Plan(M, fe.MASS, 6, precision="fp32", quad_scheme="symmetric")
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == 0
    y64 = fe.Plan(M, fe.MASS, 6, quad_scheme="symmetric").apply(cuda(u)).cpu().numpy()
    assert rel(y, y64) <= TOL32
    rng = np.random.default_rng(97)
    nodes = rng.choice(m.n_nodes, size=64, replace=False)
    cells = np.unique(np.nonzero(np.isin(m.cell2node, nodes))[0])
    o = oracle.Oracle(2, 3, 6, m.coords, m.cell2vertex[cells], m.cell2node[cells], m.n_nodes, "symmetric")
    ref = o.mass(u)
    assert np.abs(y[nodes] - ref[nodes]).max() <= TOL32 * np.abs(y64).max()
