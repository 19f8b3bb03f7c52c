"""GPU parity of the tensor-core kernel (16-bit or TF32 contractions, FP32
accumulate) against the FP64 oracle.

Stated bound.  The kernel rounds three things to the 16-bit type: the
tabulation (once, in the plan), each cell's DoFs (for gradient forms after
removing a per-cell constant) scaled by a power of two, and the pointwise
values E' after scaling; products accumulate in FP32, and geometry, the
Neo-Hookean law, the output scaling and the scatter are FP64 (the kinematic
contractions with J^{-1} FP32).  Each rounding is a relative perturbation of
at most the unit roundoff u16 (bfloat16: 2^-8 = 3.9e-3, binary16 and TF32:
2^-11 = 4.9e-4); through the two contractions they are amplified by the ratio of the
absolute terms to the result.  Measured: mass and elasticity 0.6-1.2 u16 up to
P6; the Neo-Hookean Jacobian 1-4.3 u16, largest at P6 where the linearisation
point's gradient (a smooth field) is evaluated from 16-bit data.  The stated
bounds, used as the parity tolerances, are per form and precision
(tests/precision_bounds.py: the largest measured deviation times 1.5), norm-wise
relative to ||y_ref||_inf.  A lower bound (> 1e-7) checks that the work really
ran in 16 bits.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from feinputs import structured_mesh, uniform_field

from precision_bounds import bound16, check16

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


def make(fe, dim, N, p, seed, scale=1.0):
    m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=seed)
    if scale != 1.0:
        m.coords = m.coords * scale
    return m, fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)


# (kind, dim, N, p, q, scheme): every case spans several 128-cell tiles with a ragged tail
CASES = [
    ("mass", 2, 13, 1, 2, "conical"), ("mass", 2, 13, 3, 6, "symmetric"), ("mass", 2, 13, 6, 12, "conical"),
    ("mass", 3, 5, 2, 4, "conical"), ("mass", 3, 5, 4, 8, "conical"),
    ("elasticity", 2, 13, 2, 2, "symmetric"), ("elasticity", 2, 13, 4, 6, "symmetric"),
    ("elasticity", 2, 13, 6, 10, "conical"), ("elasticity", 3, 5, 1, 0, "conical"),
    ("elasticity", 3, 5, 2, 2, "symmetric"), ("elasticity", 3, 5, 2, 2, "conical"),
    ("elasticity", 3, 5, 4, 6, "conical"), ("elasticity", 3, 5, 4, 6, "symmetric"),
]


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
@pytest.mark.parametrize("kind,dim,N,p,q,scheme", CASES)
def test_tc_parity(fe, kind, dim, N, p, q, scheme, prec):
    m, M = make(fe, dim, N, p, 300 + 10 * dim + p)
    assert m.n_cells > 256 and m.n_cells % 128 != 0
    o = oracle.Oracle.from_mesh(m, q, scheme=scheme)
    nc = 1 if kind == "mass" else dim
    u = uniform_field(m.n_nodes * nc, 7 + p)
    if kind == "mass":
        plan = fe.Plan(M, fe.MASS, q, precision=prec, quad_scheme=scheme)
        ref = o.mass(u)
    else:
        plan = fe.Plan(M, fe.ELASTICITY, q, lam=1.25, mu=1.0, precision=prec, quad_scheme=scheme)
        ref = o.elasticity(u, 1.25, 1.0)
    assert plan.info.kernel == 2
    y = plan.apply(cuda(u))
    err = rel(y, ref)
    check16(kind, prec, err, f"d{dim} N{N} p{p} q{q} {scheme}")
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
def test_tc_scale_invariance(fe, prec):
    """Per-cell power-of-two scaling: A(2^k u) = 2^k A(u) up to the order of the
    FP64 atomics, for magnitudes far outside binary16's range."""
    m, M = make(fe, 3, 5, 2, 41)
    plan = fe.Plan(M, fe.ELASTICITY, 2, lam=1.25, mu=1.0, precision=prec, quad_scheme="symmetric")
    u = uniform_field(m.n_nodes * 3, 9)
    y1 = plan.apply(cuda(u)).cpu().numpy()
    for k in (-700, -60, 40, 700):
        yk = plan.apply(cuda(u * 2.0 ** k)).cpu().numpy()
        assert np.abs(yk * 2.0 ** -k - y1).max() <= 1e-13 * np.abs(y1).max(), k
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
def test_tc_tiny_and_huge_cells(fe, prec):
    """Mesh scaled by 2^-24 and 2^+24: J^{-1} is scaled per cell by a power of
    two, so the pointwise values stay in range and the bound still holds."""
    for s in (2.0 ** -24, 2.0 ** 24):
        m, M = make(fe, 2, 13, 4, 42, scale=s)
        o = oracle.Oracle.from_mesh(m, 6, scheme="symmetric")
        u = uniform_field(m.n_nodes * 2, 10)
        plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, precision=prec, quad_scheme="symmetric")
        check16("elasticity", prec, rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0)), f"p4 2d scale {s}")
        assert plan.status() == 0


def test_tc_edge_cases(fe):
    # empty mesh: y = 0, nothing launched
    m, _ = make(fe, 2, 4, 3, 43)
    M0 = fe.Mesh(2, 3, m.coords, m.cell2vertex[:0], m.cell2node[:0], m.n_nodes)
    plan = fe.Plan(M0, fe.MASS, 6, precision="bf16")
    y = plan.apply(cuda(np.ones(m.n_nodes)))
    assert float(y.abs().max()) == 0.0
    # a single cell (one partial tile)
    M1 = fe.Mesh(2, 3, m.coords, m.cell2vertex[:1], m.cell2node[:1], m.n_nodes)
    o1 = oracle.Oracle(2, 3, 6, m.coords, m.cell2vertex[:1], m.cell2node[:1], m.n_nodes)
    u = uniform_field(m.n_nodes, 3)
    check16("mass", "fp16", rel(fe.Plan(M1, fe.MASS, 6, precision="fp16").apply(cuda(u)), o1.mass(u)),
            "one cell", floor=None)
    # accumulate: y += A u
    m, M = make(fe, 2, 13, 3, 44)
    o = oracle.Oracle.from_mesh(m, 6)
    u = uniform_field(m.n_nodes, 4)
    y0 = uniform_field(m.n_nodes, 5)
    acc = fe.Plan(M, fe.MASS, 6, precision="fp16", accumulate=True)
    y = acc.apply(cuda(u), cuda(y0.copy()))
    ref = y0 + o.mass(u)
    assert np.abs(y.cpu().numpy() - ref).max() <= bound16("mass", "fp16") * np.abs(o.mass(u)).max()
    # forms without a tensor-core variant are refused
    with pytest.raises(Exception):
        fe.Plan(M, fe.NH_RESIDUAL, 6, mu=1.0, lam=1.0, precision="bf16")
    with pytest.raises(Exception):
        fe.Plan(M, fe.SVK_RESIDUAL, 6, mu=1.0, lam=1.0, precision="fp16")


def test_tc_bad_index_sets_status(fe):
    """An out-of-range node index skips its cell and reports FE_ERR_INDEX; the
    other cells are still applied."""
    from paper_2506_17471_gb300 import _native as N
    m, _ = make(fe, 2, 13, 3, 45)
    c2n = m.cell2node.copy()
    c2n[200, 4] = m.n_nodes + 7
    M = fe.Mesh(2, 3, m.coords, m.cell2vertex, c2n, m.n_nodes)
    plan = fe.Plan(M, fe.MASS, 6, precision="bf16")
    u = uniform_field(m.n_nodes, 6)
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == N.FE_ERR_INDEX
    keep = np.ones(m.n_cells, dtype=bool)
    keep[200] = False
    o = oracle.Oracle(2, 3, 6, m.coords, m.cell2vertex[keep], m.cell2node[keep], m.n_nodes)
    check16("mass", "bf16", rel(y, o.mass(u)), "bad index", floor=None)
    assert plan.status() == 0


def test_tc_conversions_match_hardware(fe):
    """The exact integer binary64 -> 16-bit conversions agree bit for bit with
    CUDA's __double2bfloat16 / __double2half, and the kernel's rounding pass
    (rounding to odd into binary32, then the hardware conversion) agrees bit for
    bit with them (and with the TF32 one) at several power-of-two scales."""
    from paper_2506_17471_gb300 import _native as N
    rng = np.random.default_rng(1)
    vals = [rng.standard_normal(300_000) * 2.0 ** rng.integers(-150, 140, 300_000),
            rng.uniform(-1, 1, 100_000),
            np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 65504.0, 65520.0, 65519.99, 6e-8, 2.0 ** -25,
                      2.0 ** -25 * 1.0000001, 3.3895313892515355e38, 3.39e38, 1e-300, 5e-324])]
    h = rng.standard_normal(100_000).astype(np.float16)
    hn = np.nextafter(h, np.float16(np.inf))
    vals.append((h.astype(np.float64) + hn.astype(np.float64)) / 2)   # binary16 ties
    x = cuda(np.concatenate(vals))
    count = torch.zeros(3, dtype=torch.int64, device="cuda")
    assert N.lib.fe_selftest_conversions16(ctypes.c_void_p(x.data_ptr()), x.numel(),
                                           ctypes.c_void_p(count.data_ptr()), None) == 0
    assert count.tolist() == [0, 0, 0]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_full_mass_p3_2d(fe, prec):
    """hp-sweep size: mass P3 on 2 x 667^2 triangles (4,008,004 DoFs), all outputs."""
    m, M = make(fe, 2, 667, 3, 20250620)
    o = oracle.Oracle.from_mesh(m, 6, scheme="symmetric")
    u = uniform_field(m.n_nodes, 21)
    plan = fe.Plan(M, fe.MASS, 6, precision=prec, quad_scheme="symmetric")
    check16("mass", prec, rel(plan.apply(cuda(u)), o.mass(u, threads=16)), "p3 2d N667")
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
def test_tc_full_elasticity_p4_3d(fe, prec):
    """hp-sweep size: elasticity P4 on 6 x 27^3 tetrahedra (3,885,087 DoFs), all outputs."""
    m, M = make(fe, 3, 27, 4, 20250622)
    o = oracle.Oracle.from_mesh(m, 6)
    u = uniform_field(m.n_nodes * 3, 22)
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, precision=prec)
    check16("elasticity", prec, rel(plan.apply(cuda(u)), o.elasticity(u, 1.25, 1.0, threads=16)), "p4 3d N27")
    assert plan.status() == 0


NH_CASES = [(2, 13, 2, 4), (2, 13, 4, 8), (2, 13, 6, 12), (3, 5, 2, 4)]


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
@pytest.mark.parametrize("dim,N,p,q", NH_CASES)
def test_tc_nh_jacobian(fe, dim, N, p, q, prec):
    """Neo-Hookean Jacobian action: u_lin and du both in 16 bits (each scaled per
    cell by its own power of two), tangent dP/dF, log det F and pull-back in
    FP64, per-cell P0 Lame parameters."""
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, dim, N, p, 500 + 10 * dim + p)
    assert m.n_cells > 256 and m.n_cells % 128 != 0
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 3)
    ul = sinusoid_displacement(m, 4)
    du = uniform_field(m.n_nodes * dim, 5)
    plan = fe.Plan(M, fe.NH_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision=prec)
    assert plan.info.kernel == 2
    err = rel(plan.apply(cuda(du)), o.nh_jacobian(ul, du, mu, lam))
    check16("nh_jacobian", prec, err, f"d{dim} N{N} p{p} q{q}")
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_full_nh_jacobian_p6_2d(fe, prec):
    """hp-sweep size: Neo-Hookean Jacobian action P6 on 2 x 236^2 triangles
    (4,015,778 DoFs), quadrature degree 12, all outputs."""
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, 2, 236, 6, 20250621)
    o = oracle.Oracle.from_mesh(m, 12)
    mu, lam = lame_fields(m.n_cells, 2)
    ul = sinusoid_displacement(m, 3)
    du = uniform_field(m.n_nodes * 2, 4)
    plan = fe.Plan(M, fe.NH_JACOBIAN, 12, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision=prec)
    check16("nh_jacobian", prec, rel(plan.apply(cuda(du)), o.nh_jacobian(ul, du, mu, lam, threads=16)),
            "p6 2d N236")
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
def test_tc_material_scaling(fe, prec):
    """Lame parameters far from O(1) (and conical rules with very small weights):
    E' is scaled per plan / per cell by powers of two, so binary16 neither
    overflows nor loses precision in its subnormal range."""
    m, M = make(fe, 3, 5, 3, 46)
    o = oracle.Oracle.from_mesh(m, 4)
    u = uniform_field(m.n_nodes * 3, 11)
    for lam, mu in ((3.0e4, 2.0e4), (2.0e-5, 1.0e-5)):
        plan = fe.Plan(M, fe.ELASTICITY, 4, lam=lam, mu=mu, precision=prec)
        check16("elasticity", prec, rel(plan.apply(cuda(u)), o.elasticity(u, lam, mu)), f"lam {lam}")
        assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("kind,dim,N,p,q", [("laplace", 2, 13, 2, 2), ("laplace", 2, 13, 4, 6),
                                            ("laplace", 3, 5, 3, 4), ("helmholtz", 2, 13, 4, 8),
                                            ("helmholtz", 3, 5, 2, 4), ("helmholtz", 3, 5, 4, 8)])
def test_tc_laplace_helmholtz(fe, kind, dim, N, p, q, prec):
    """Scalar gradient forms on the tensor cores: the Laplacian with the per-cell
    shift, Helmholtz with its value row (no shift: values need the constant)."""
    m, M = make(fe, dim, N, p, 600 + 10 * dim + p)
    assert m.n_cells % 128 != 0
    o = oracle.Oracle.from_mesh(m, q)
    u = uniform_field(m.n_nodes, 12 + p)
    if prec == "tf32" and (kind, dim, p, q) == ("helmholtz", 3, 4, 8):
        # 4-byte operands: the 125-point tables exceed shared memory, refused cleanly
        with pytest.raises(fe.FeError) as e:
            fe.Plan(M, fe.HELMHOLTZ, q, precision=prec)
        assert e.value.code == 2
        return
    plan = fe.Plan(M, getattr(fe, kind.upper()), q, precision=prec)
    assert plan.info.kernel == 2
    err = rel(plan.apply(cuda(u)), getattr(o, kind)(u))
    check16(kind, prec, err, f"d{dim} N{N} p{p} q{q}")
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
def test_tc_helmholtz_cell_scale(fe, prec):
    """Helmholtz mixes a value term (scale h^d) and a gradient term (h^(d-2)); both
    share the per-cell output factor, on meshes scaled by 2^-20 and 2^+20."""
    for s in (2.0 ** -20, 2.0 ** 20):
        m, M = make(fe, 2, 13, 3, 47, scale=s)
        o = oracle.Oracle.from_mesh(m, 6)
        u = uniform_field(m.n_nodes, 13)
        plan = fe.Plan(M, fe.HELMHOLTZ, 6, precision=prec)
        check16("helmholtz", prec, rel(plan.apply(cuda(u)), o.helmholtz(u)), f"p3 2d scale {s}")
        assert plan.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32"])
@pytest.mark.parametrize("dim,N,p,q", [(2, 13, 2, 4), (2, 13, 4, 8), (3, 5, 2, 4)])
def test_tc_svk_jacobian(fe, dim, N, p, q, prec):
    """St. Venant-Kirchhoff Jacobian action (the paper's hyperelastic law) on the
    tensor cores: two 16-bit fields, FP64 law."""
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, dim, N, p, 800 + 10 * dim + p)
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 3)
    ul = sinusoid_displacement(m, 4)
    du = uniform_field(m.n_nodes * dim, 5)
    plan = fe.Plan(M, fe.SVK_JACOBIAN, q, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision=prec)
    assert plan.info.kernel == 2
    err = rel(plan.apply(cuda(du)), o.svk_jacobian(ul, du, mu, lam))
    check16("svk_jacobian", prec, err, f"d{dim} N{N} p{p} q{q}")
    assert plan.status() == 0


TOL_X2 = 5e-5   # split binary16 operands: the FP32 bound


@pytest.mark.parametrize("kind,dim,N,p,q", [("mass", 2, 13, 3, 6), ("elasticity", 3, 5, 2, 2),
                                            ("elasticity", 3, 5, 4, 6), ("laplace", 2, 13, 4, 6),
                                            ("helmholtz", 3, 5, 3, 6), ("elasticity", 2, 13, 6, 10)])
def test_tc_fp16x2(fe, kind, dim, N, p, q):
    """Split binary16 operands (hi + lo) with three tensor-core products per term:
    error of the FP32 class, far below the single 16-bit rounding."""
    m, M = make(fe, dim, N, p, 900 + 10 * dim + p)
    o = oracle.Oracle.from_mesh(m, q)
    nc = 1 if kind in ("mass", "laplace", "helmholtz") else dim
    u = uniform_field(m.n_nodes * nc, 14 + p)
    kw = dict(lam=1.25, mu=1.0) if kind == "elasticity" else {}
    plan = fe.Plan(M, getattr(fe, kind.upper()), q, precision="fp16x2", **kw)
    assert plan.info.kernel == 2
    ref = o.elasticity(u, 1.25, 1.0) if kind == "elasticity" else getattr(o, kind)(u)
    err = rel(plan.apply(cuda(u)), ref)
    assert 1e-10 < err <= TOL_X2, err
    assert plan.status() == 0


def test_tc_fp16x2_nh_jacobian(fe):
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, 2, 13, 4, 950)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 3)
    ul = sinusoid_displacement(m, 4)
    du = uniform_field(m.n_nodes * 2, 5)
    plan = fe.Plan(M, fe.NH_JACOBIAN, 8, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision="fp16x2")
    assert rel(plan.apply(cuda(du)), o.nh_jacobian(ul, du, mu, lam)) <= TOL_X2
    assert plan.status() == 0


def test_tc_fp16x2_tables_too_large(fe):
    """The split operands double the staged basis tables; Helmholtz P4 3D with 125
    quadrature points then exceeds shared memory and the plan is refused cleanly."""
    m, M = make(fe, 3, 3, 4, 960)
    with pytest.raises(fe.FeError) as e:
        fe.Plan(M, fe.HELMHOLTZ, 8, precision="fp16x2")
    assert e.value.code == 2
    assert fe.Plan(M, fe.HELMHOLTZ, 8, precision="fp16").info.kernel == 2


@pytest.mark.parametrize("prec", ["fp16", "fp16x2"])
@pytest.mark.parametrize("kind,dim,N,p,q", [("elasticity", 3, 5, 4, 6), ("mass", 2, 13, 3, 6),
                                            ("nh_jacobian", 2, 13, 4, 8)])
def test_tc_pipelines_and_threads_per_cell(fe, kind, dim, N, p, q, prec):
    """Every launch shape gives the same result to rounding: the automatic layout
    (the most pipelines that fit, then 2 or 4 threads per cell when fewer than
    four pipelines fit) and each forced pipeline count (one thread per cell)."""
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, dim, N, p, 970 + 10 * dim + p)
    o = oracle.Oracle.from_mesh(m, q)
    nc = 1 if kind == "mass" else dim
    u = uniform_field(m.n_nodes * nc, 21 + p)
    kw, ref = {}, None
    if kind == "elasticity":
        kw = dict(lam=1.25, mu=1.0)
        ref = o.elasticity(u, 1.25, 1.0)
    elif kind == "mass":
        ref = o.mass(u)
    else:
        mu, lam = lame_fields(m.n_cells, 5)
        ul = sinusoid_displacement(m, 6)
        kw = dict(mu_cell=mu, lam_cell=lam, u_lin=cuda(ul))
        ref = o.nh_jacobian(ul, u, mu, lam)
    tol = TOL_X2 if prec == "fp16x2" else bound16(kind, prec)
    auto = fe.Plan(M, getattr(fe, kind.upper()), q, precision=prec, **kw)
    y_auto = auto.apply(cuda(u))
    assert rel(y_auto, ref) <= tol and auto.status() == 0
    tpb = auto.info.threads_per_block
    assert tpb in (128, 256, 512) and auto.info.kernel == 2
    shapes = 0
    for tc in (128, 256, 512):
        try:
            plan = fe.Plan(M, getattr(fe, kind.upper()), q, precision=prec, tile_cells=tc, **kw)
        except fe.FeError as e:
            assert e.code == 2   # that many pipelines do not fit this layout
            continue
        assert plan.info.threads_per_block == tc
        y = plan.apply(cuda(u))
        assert rel(y, ref) <= tol and plan.status() == 0
        # the same rounded operands; the chunking of the quadrature points (and so the
        # FP32 accumulation order) and the scatter order may differ
        assert rel(y, y_auto.cpu().numpy()) <= 1e-5
        shapes += 1
    assert shapes >= 1
    with pytest.raises(fe.FeError):
        fe.Plan(M, getattr(fe, kind.upper()), q, precision=prec, tile_cells=384, **kw)


@pytest.mark.parametrize("j", [3, 30])
def test_tc_bad_index_two_threads_per_cell(fe, j):
    """Elasticity P4 3D runs two threads per cell, each gathering half of the cell's
    node batches: a bad index in either half (local node 3: the first thread's
    batch; 30: the second's) must skip the whole cell on both threads."""
    from paper_2506_17471_gb300 import _native as N
    m, _ = make(fe, 3, 5, 4, 46)
    c2n = m.cell2node.copy()
    c2n[300, j] = -5
    M = fe.Mesh(3, 4, m.coords, m.cell2vertex, c2n, m.n_nodes)
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, precision="fp16")
    assert plan.info.threads_per_block == 512
    u = uniform_field(m.n_nodes * 3, 7)
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == N.FE_ERR_INDEX
    keep = np.ones(m.n_cells, dtype=bool)
    keep[300] = False
    o = oracle.Oracle(3, 4, 6, m.coords, m.cell2vertex[keep], m.cell2node[keep], m.n_nodes)
    check16("elasticity", "fp16", rel(y, o.elasticity(u, 1.25, 1.0)), "bad index 2 threads", floor=None)


@pytest.mark.parametrize("bad", ["vertex", "degenerate"])
def test_tc_shared_geometry_invalid_cell(fe, bad):
    """With two threads per cell the cell's first thread computes the geometry and
    hands it to the second: an out-of-range vertex index (FE_ERR_INDEX) or a
    degenerate cell (FE_ERR_BAD_MESH) must skip the whole cell on both threads,
    and every other cell (their geometry shared the same way) is applied."""
    from paper_2506_17471_gb300 import _native as N
    m, _ = make(fe, 3, 5, 4, 47)
    c2v = m.cell2vertex.copy()
    if bad == "vertex":
        c2v[310, 2] = m.coords.shape[0] + 11
    else:
        c2v[310, 3] = c2v[310, 1]                  # the cell collapses onto a face
    M = fe.Mesh(3, 4, m.coords, c2v, m.cell2node, m.n_nodes)
    plan = fe.Plan(M, fe.ELASTICITY, 6, lam=1.25, mu=1.0, precision="fp16")
    assert plan.info.threads_per_block == 512
    u = uniform_field(m.n_nodes * 3, 8)
    y = plan.apply(cuda(u)).cpu().numpy()
    assert plan.status() == (N.FE_ERR_INDEX if bad == "vertex" else N.FE_ERR_BAD_MESH)
    keep = np.ones(m.n_cells, dtype=bool)
    keep[310] = False
    o = oracle.Oracle(3, 4, 6, m.coords, m.cell2vertex[keep], m.cell2node[keep], m.n_nodes)
    check16("elasticity", "fp16", rel(y, o.elasticity(u, 1.25, 1.0)), "shared geometry " + bad, floor=None)


@pytest.mark.parametrize("kind", ["nh_jacobian", "svk_jacobian"])
@pytest.mark.parametrize("dim,N,p,q", [(2, 13, 3, 6), (3, 5, 2, 4)])
def test_tc_fp16x2_hyperelastic(fe, kind, dim, N, p, q):
    """Split binary16 operands for both hyperelastic Jacobian actions, 2D and 3D:
    the FP32-class bound although the law stays FP64 and the linearisation
    point is a smooth field."""
    from feinputs import lame_fields
    from feinputs.fields import sinusoid_displacement
    m, M = make(fe, dim, N, p, 990 + 10 * dim + p)
    o = oracle.Oracle.from_mesh(m, q)
    mu, lam = lame_fields(m.n_cells, 8)
    ul = sinusoid_displacement(m, 9)
    du = uniform_field(m.n_nodes * dim, 10)
    plan = fe.Plan(M, getattr(fe, kind.upper()), q, mu_cell=mu, lam_cell=lam, u_lin=cuda(ul), precision="fp16x2")
    assert plan.info.kernel == 2
    ref = getattr(o, kind)(ul, du, mu, lam)
    assert rel(plan.apply(cuda(du)), ref) <= TOL_X2
    assert plan.status() == 0


def test_tc_node_limit(fe):
    """The tensor-core kernel serves every tabulated degree (up to 10) with at most
    256 local nodes: P9 tetrahedra (220 nodes) plan and run, P10 tetrahedra (286)
    are refused cleanly.  (At P9 the equispaced basis amplifies the 16-bit operand
    rounding by its Lebesgue constant, so only the launch and a loose bound against
    the FP64 kernel are checked here; accuracy is pinned up to P6.)"""
    m, M = make(fe, 3, 2, 9, 991)
    u = uniform_field(m.n_nodes, 11)
    plan = fe.Plan(M, fe.MASS, 2, precision="fp16")
    assert plan.info.n_loc == 220 and plan.info.kernel == 2
    y = plan.apply(cuda(u))
    assert plan.status() == 0 and bool(torch.isfinite(y).all())
    # against the FP64 cells-per-CTA kernel (the oracle stops below this degree)
    y64 = fe.Plan(M, fe.MASS, 2).apply(cuda(u)).cpu().numpy()
    assert rel(y, y64) <= 0.1
    m2, M2 = make(fe, 3, 1, 10, 992)
    with pytest.raises(fe.FeError) as e:
        fe.Plan(M2, fe.MASS, 2, precision="fp16")
    assert e.value.code == 2


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_benchmark_workload_elasticity_p4_3d_n27(fe, prec):
    """The hp-sweep workload as the benchmark builds it (24-point fully symmetric
    degree-6 rule) on the tensor cores: every output against the oracle."""
    from feinputs.workloads import ELASTICITY_P4_3D_N27 as wl
    m = wl.mesh()
    M = fe.Mesh(3, wl.degree, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
    u = wl.field(m)
    o = oracle.Oracle.from_mesh(m, wl.quad_degree, scheme=wl.quad_scheme)
    plan = fe.Plan(M, fe.ELASTICITY, wl.quad_degree, lam=wl.lam, mu=wl.mu, precision=prec,
                   quad_scheme=wl.quad_scheme)
    assert plan.info.kernel == 2 and plan.info.nq == 24
    check16("elasticity", prec, rel(plan.apply(cuda(u)), o.elasticity(u, wl.lam, wl.mu, threads=16)),
            "p4 3d N27 24-point rule")
    assert plan.status() == 0
