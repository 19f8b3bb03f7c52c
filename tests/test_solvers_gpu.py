"""GPU tests of CG and of FP64 iterative refinement around the FP32-contraction action.

Right-hand sides come from the oracle (b = A_oracle x* on the CPU), and the
converged solutions are checked with the oracle's own action: the true relative
residual ||M (b - A_oracle x)|| / ||M b|| must be <= 1e-10 (the refinement
target) up to the FP64 rounding of the oracle's action.
"""

import numpy as np
import pytest
import torch

import oracle
from feinputs import structured_mesh, uniform_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_17471_gb300 as fe
    from paper_2506_17471_gb300 import solvers
    return fe, solvers


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_cg_mass_fp64_and_refined_fp32(fe):
    fe, solvers = fe
    m = structured_mesh(2, 24, 3, jitter=0.2, seed=1)
    o = oracle.Oracle.from_mesh(m, 6)
    xs = uniform_field(m.n_nodes, 2)
    b = o.mass(xs)
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    p64 = fe.Plan(M, fe.MASS, 6)
    p32 = fe.Plan(M, fe.MASS, 6, precision="fp32")
    bt = cuda(b)
    x, st = solvers.cg(lambda u, y: p64.apply(u, y), bt, rtol=1e-10)
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - o.mass(xh)) <= 1.5e-10 * np.linalg.norm(b)
    assert st.iterations > 0
    x2, st2 = solvers.cg_ir(lambda u, y: p64.apply(u, y), lambda u, y: p32.apply(u, y), bt, tol=1e-10)
    xh2 = x2.cpu().numpy()
    assert st2.rel_residual <= 1e-10
    assert np.linalg.norm(b - o.mass(xh2)) <= 1.5e-10 * np.linalg.norm(b)
    assert np.abs(xh2 - xs).max() <= 1e-6 * np.abs(xs).max()


def test_cg_ir_elasticity_dirichlet(fe):
    fe, solvers = fe
    m = structured_mesh(3, 6, 2, jitter=0.15, seed=3)
    o = oracle.Oracle.from_mesh(m, 2)
    free = np.repeat(~m.boundary_nodes(), 3).astype(np.uint8)
    xs = uniform_field(m.n_nodes * 3, 4) * free
    b = free * o.elasticity(xs, 1.25, 1.0)
    M = fe.Mesh(3, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    p64 = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0)
    p32 = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0, precision="fp32")
    mask = cuda(free)
    x, st = solvers.cg_ir(lambda u, y: p64.apply(u, y), lambda u, y: p32.apply(u, y), cuda(b), mask,
                          tol=1e-10)
    xh = x.cpu().numpy()
    assert st.rel_residual <= 1e-10 and st.outer >= 1
    assert np.all(xh[free == 0] == 0.0)
    res = free * (b - o.elasticity(xh, 1.25, 1.0))
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(b)
    # plain FP64 CG on the same system reaches the same accuracy
    x64, st64 = solvers.cg(lambda u, y: p64.apply(u, y), cuda(b), mask, rtol=1e-10)
    res64 = free * (b - o.elasticity(x64.cpu().numpy(), 1.25, 1.0))
    assert np.linalg.norm(res64) <= 1.5e-10 * np.linalg.norm(b)


def test_vector_kernels_deterministic(fe):
    fe, solvers = fe
    n = 1_000_003
    x = torch.rand(n, dtype=torch.float64, device="cuda")
    y = torch.rand(n, dtype=torch.float64, device="cuda")
    w = solvers.Workspace(n, x.device)
    d1 = w.dot(x, y)
    d2 = w.dot(x, y)
    assert d1 == d2                                   # bitwise reproducible
    ref = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
    assert abs(d1 - ref) <= 1e-12 * abs(ref)
    mask = (torch.rand(n, device="cuda") > 0.5).to(torch.uint8)
    dm = w.dot(x, y, mask)
    refm = float(np.dot(x.cpu().numpy() * mask.cpu().numpy(), y.cpu().numpy()))
    assert abs(dm - refm) <= 1e-12 * abs(refm)
