"""fe_action_noalloc: the action for callers that cannot allocate device memory.

Callers whose device memory is owned up front by their own pool allocator, or
that may not call cudaMalloc after start-up, cannot create a plan.  This entry
point runs the same kernel with its scratch in a static device array of the
library.  The test calls it through the C-ABI twice in a row, with different
forms and table sizes (the array keeps the previous call's contents), and checks
each output against fe_action's within the parity tolerance of the suite; a
second test passes page-locked tables and overwrites them as soon as the call
returns.
This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""

import ctypes

import numpy as np
import pytest
import torch

from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2506_17471_gb300 as fe
    assert torch.cuda.is_available()
    return fe


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def call_noalloc(fe, plan, u, y):
    """fe_action_noalloc with the plan's own mesh/form descriptors and host tables."""
    from paper_2506_17471_gb300 import _native as N
    mesh = plan.mesh
    _, wts, tab = fe.tabulate(mesh.dim, mesh.degree, plan._form.quad_degree)
    tab = np.ascontiguousarray(tab)
    wts = np.ascontiguousarray(wts)
    status = ctypes.c_int(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = N.lib.fe_action_noalloc(ctypes.byref(plan._form), ctypes.byref(plan._mesh_c),
                                 tab.ctypes.data_as(ctypes.c_void_p),
                                 wts.ctypes.data_as(ctypes.c_void_p), int(len(wts)),
                                 ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.byref(status), stream)
    return rc, status.value


def test_noalloc_matches_fe_action_on_two_calls_in_a_row(fe):
    # call 1: elasticity P2 tets (8-point rule, 328-double table)
    m3 = structured_mesh(3, 5, 2, jitter=0.15, seed=81)
    M3 = fe.Mesh(3, 2, m3.coords, m3.cell2vertex, m3.cell2node, m3.n_nodes)
    p3 = fe.Plan(M3, fe.ELASTICITY, 2, lam=1.25, mu=1.0)
    u3 = torch.from_numpy(uniform_field(m3.n_nodes * 3, 82)).cuda()
    y3 = torch.full_like(u3, 3.0)          # stale contents must be overwritten
    rc, st = call_noalloc(fe, p3, u3, y3)
    assert (rc, st) == (0, 0)
    assert rel(y3, p3.apply(u3)) <= TOL

    # call 2: Neo-Hookean residual P4 triangles, per-cell coefficients
    # (25-point rule, 1150-double table; the array still holds call 1's table)
    m2 = structured_mesh(2, 9, 4, jitter=0.2, seed=83)
    M2 = fe.Mesh(2, 4, m2.coords, m2.cell2vertex, m2.cell2node, m2.n_nodes)
    mu, lam = lame_fields(m2.n_cells, 84)
    p2 = fe.Plan(M2, fe.NH_RESIDUAL, 8, mu_cell=mu, lam_cell=lam)
    u2 = torch.from_numpy(sinusoid_displacement(m2, 85)).cuda()
    y2 = torch.full_like(u2, -1.0)
    rc, st = call_noalloc(fe, p2, u2, y2)
    assert (rc, st) == (0, 0)
    assert rel(y2, p2.apply(u2)) <= TOL


def test_noalloc_reads_page_locked_tables_before_returning(fe):
    """Tables in page-locked host memory are copied asynchronously; the entry
    point waits for its copies, so overwriting the tables as soon as it returns
    (before the stream is synchronised) must not change the result."""
    m = structured_mesh(3, 5, 2, jitter=0.15, seed=86)
    M = fe.Mesh(3, 2, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0)
    _, wts, tab = fe.tabulate(3, 2, 2)
    tab_p = torch.from_numpy(np.ascontiguousarray(tab)).pin_memory()
    wts_p = torch.from_numpy(np.ascontiguousarray(wts)).pin_memory()
    u = torch.from_numpy(uniform_field(m.n_nodes * 3, 87)).cuda()
    y = torch.empty_like(u)
    ref = plan.apply(u)
    torch.cuda.synchronize()
    for _ in range(2):
        rc = call_noalloc_async(fe, plan, u, y, tab_p, wts_p)
        assert rc == 0
        tab_p.fill_(1e300)      # the caller reuses its buffers right away
        wts_p.fill_(-1e300)
        torch.cuda.synchronize()
        assert rel(y, ref) <= TOL
        tab_p.copy_(torch.from_numpy(np.ascontiguousarray(tab)))
        wts_p.copy_(torch.from_numpy(np.ascontiguousarray(wts)))


def call_noalloc_async(fe, plan, u, y, tab_p, wts_p):
    """fe_action_noalloc from page-locked tables, without the status read-back
    (which would synchronise the stream)."""
    from paper_2506_17471_gb300 import _native as N
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return N.lib.fe_action_noalloc(ctypes.byref(plan._form), ctypes.byref(plan._mesh_c),
                                   ctypes.c_void_p(tab_p.data_ptr()), ctypes.c_void_p(wts_p.data_ptr()),
                                   int(wts_p.numel()), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), None, stream)


def test_noalloc_rejects_tables_beyond_its_scratch(fe):
    from paper_2506_17471_gb300 import _native as N
    m = structured_mesh(2, 2, 6)
    M = fe.Mesh(2, 6, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    form = N.FeForm(N.FE_FORM_MASS, 24, N.FE_PREC_FP64, 0, 0.0, 0.0, 0, 0, 0)
    mesh_c = M._c()
    _, wts, tab = fe.tabulate(2, 6, 24)       # 169 points x 3 x 28 + 169 > 12288 doubles
    tab, wts = np.ascontiguousarray(tab), np.ascontiguousarray(wts)
    u = torch.ones(m.n_nodes, dtype=torch.float64, device="cuda")
    y = torch.empty_like(u)
    rc = N.lib.fe_action_noalloc(ctypes.byref(form), ctypes.byref(mesh_c),
                                 tab.ctypes.data_as(ctypes.c_void_p),
                                 wts.ctypes.data_as(ctypes.c_void_p), int(len(wts)),
                                 ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 None, None)
    assert rc == 1  # FE_ERR_INVALID_ARG, nothing launched
