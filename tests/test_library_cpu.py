"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol
that include/feaction.h declares, its host tabulation (S0 of the hot path)
matches the oracle's independent tabulation, and argument validation rejects bad
input before anything reaches CUDA."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2506_17471_gb300 as fe
    return fe


def declared_functions():
    with open(os.path.join(ROOT, "include", "feaction.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(fe):
    from paper_2506_17471_gb300 import _native
    names = declared_functions()
    assert names, "no declarations found"
    assert set(names) == set(_native.EXPORTS)
    lib = ctypes.CDLL(fe.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(fe):
    from paper_2506_17471_gb300 import _native
    for code, name in _native.STATUS_NAMES.items():
        assert _native.lib.fe_status_string(code).decode() == name
    assert _native.lib.fe_status_string(999).decode() == "FE_ERR_UNKNOWN"


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("degree", [1, 2, 4, 6])
@pytest.mark.parametrize("q", [0, 2, 4, 8, 12, 17])
def test_tabulate_matches_oracle(fe, dim, degree, q):
    import oracle
    if dim == 3 and degree == 6 and q > 12:
        pytest.skip("large")
    pts, wts, tab = fe.tabulate(dim, degree, q)
    p2, w2, t2 = oracle.tabulate(dim, degree, q)
    assert pts.shape == p2.shape and tab.shape == t2.shape
    np.testing.assert_allclose(pts, p2, rtol=0, atol=1e-15)  # a few ulps of points in [0, 1]
    np.testing.assert_allclose(wts, w2, rtol=1e-14, atol=1e-17)
    assert np.abs(tab - t2).max() <= 1e-13 * np.abs(t2).max()


def test_tabulate_rejects_bad_arguments(fe):
    from paper_2506_17471_gb300 import _native
    nq = ctypes.c_int(0)
    lib = _native.lib
    assert lib.fe_tabulate(4, 1, 2, ctypes.byref(nq), None, None, None, 0) == 1
    assert lib.fe_tabulate(2, 0, 2, ctypes.byref(nq), None, None, None, 0) == 1
    assert lib.fe_tabulate(2, 1, -1, ctypes.byref(nq), None, None, None, 0) == 1
    assert lib.fe_tabulate(2, 1, 2, None, None, None, None, 0) == 1
    # too-small capacity
    buf = np.zeros(4)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    assert lib.fe_tabulate(2, 2, 4, ctypes.byref(nq), p, p, p, 4) == 1


def test_plan_create_validates_before_cuda(fe):
    from paper_2506_17471_gb300 import _native as N
    h = ctypes.c_void_p(0)
    mesh = N.FeMesh(2, 2, 4, 2, 9, 0, 0, 0)  # null arrays with cells > 0
    form = N.FeForm(N.FE_FORM_MASS, 4, 0, 0, 0.0, 0.0, 0, 0, 0)
    assert N.lib.fe_plan_create(ctypes.byref(form), ctypes.byref(mesh), ctypes.byref(h)) == 1
    mesh = N.FeMesh(4, 2, 4, 0, 9, 0, 0, 0)   # dim 4
    assert N.lib.fe_plan_create(ctypes.byref(form), ctypes.byref(mesh), ctypes.byref(h)) == 1
    mesh = N.FeMesh(2, 2, 4, 0, 9, 0, 0, 0)
    bad_kind = N.FeForm(9, 4, 0, 0, 0.0, 0.0, 0, 0, 0)
    assert N.lib.fe_plan_create(ctypes.byref(bad_kind), ctypes.byref(mesh), ctypes.byref(h)) == 1
    jac_no_lin = N.FeForm(N.FE_FORM_NH_JACOBIAN, 4, 0, 0, 0.0, 0.0, 0, 0, 0)
    assert N.lib.fe_plan_create(ctypes.byref(jac_no_lin), ctypes.byref(mesh), ctypes.byref(h)) == 1
    prec = N.FeForm(N.FE_FORM_MASS, 4, 7, 0, 0.0, 0.0, 0, 0, 0)
    assert N.lib.fe_plan_create(ctypes.byref(prec), ctypes.byref(mesh), ctypes.byref(h)) == 2
    assert N.lib.fe_plan_create(None, ctypes.byref(mesh), ctypes.byref(h)) == 1
    assert N.lib.fe_action(None, None, None, None) == 1
    assert N.lib.fe_plan_destroy(None) == 0


@pytest.mark.parametrize("dim,q", [(2, 2), (2, 4), (2, 6), (2, 8), (3, 2), (3, 4), (3, 5), (3, 6), (3, 7)])
@pytest.mark.parametrize("degree", [1, 2, 4])
def test_symmetric_tabulation_matches_oracle(fe, dim, q, degree):
    import oracle
    pts, wts, tab = fe.tabulate(dim, degree, q, "symmetric")
    p2, w2, t2 = oracle.tabulate(dim, degree, q, "symmetric")
    if (dim, q) in ((3, 7),):   # no tabulated symmetric rule: the conical-product fallback
        np.testing.assert_allclose(pts, p2, rtol=0, atol=1e-15)
        np.testing.assert_allclose(wts, w2, rtol=1e-14)
    else:
        # Both sides polish the rule in extended precision and round once.  The
        # results agree to the last bit except where extended precision cannot
        # settle the rounding: on x86 (64-bit long double significand) the
        # library's degree-6 tetrahedron rule has one weight one ulp below the
        # correctly rounded value (0.00167953517588677382..., which lies 0.62 ulp
        # above the lower neighbour; a 40-digit solve confirms the oracle's
        # rounding).  Both rules meet the moment equations to the same 1e-15.
        assert np.abs(np.spacing(np.abs(wts)) ** -1 * (wts - w2)).max() <= 1.0
        assert np.abs(np.spacing(np.abs(pts)) ** -1 * (pts - p2)).max() <= 1.0
    assert np.abs(tab - t2).max() <= 1e-14 * np.abs(t2).max()


# ---------------------------------------------------------------- 16-bit rounding of the tables
def _round_ref(x: float, p: int, emin: int, emax: int) -> float:
    """Round-to-nearest-even of x to a binary format with p significand bits and
    normal exponents emin..emax (IEEE 754 definition, exact rational arithmetic)."""
    from fractions import Fraction
    import math
    if math.isnan(x) or math.isinf(x) or x == 0.0:
        return x
    fx = Fraction(x)
    e = math.frexp(abs(x))[1] - 1          # 2^e <= |x| < 2^(e+1)
    q = Fraction(2) ** (max(e, emin) - (p - 1))   # quantum (subnormal below emin)
    r = round(fx / q) * q                  # round() on Fraction: ties to even
    big = (2 - Fraction(2) ** (1 - p)) * Fraction(2) ** emax
    half_ulp_max = Fraction(2) ** (emax - p)
    if abs(fx) >= big + half_ulp_max:
        return math.copysign(math.inf, x)
    return math.copysign(float(r), x) if r != 0 else math.copysign(0.0, x)


def _bits_bf16(v: float) -> int:
    return int(np.array([v], dtype=np.float32).view(np.uint32)[0] >> 16)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_round16_matches_ieee_definition(fe, prec):
    """fe_round16 (the plans' table rounding, shared with the kernel's DoF
    conversion) against round-to-nearest-even written from its definition,
    on random magnitudes, exact ties, the overflow and subnormal edges."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    rng = np.random.default_rng(11)
    p, emin, emax = (8, -126, 127) if prec == "bf16" else (11, -14, 15)
    x = list(rng.standard_normal(3000) * 2.0 ** rng.integers(emin - 14, emax + 2, 3000))
    # exact ties between neighbours and just off them
    for _ in range(1500):
        e = int(rng.integers(emin - 8, emax))
        m = int(rng.integers(2 ** (p - 1), 2 ** p))
        t = (m + 0.5) * 2.0 ** (e - p + 1)
        x += [t, -t, np.nextafter(t, 0), np.nextafter(t, np.inf)]
    big = (2 - 2.0 ** (1 - p)) * 2.0 ** emax
    x += [0.0, -0.0, np.inf, -np.inf, big, big + 2.0 ** (emax - p), np.nextafter(big + 2.0 ** (emax - p), 0),
          2.0 ** (emin - p + 1), 2.0 ** (emin - p), np.nextafter(2.0 ** (emin - p), 1), 1e-300, 5e-324]
    x = np.asarray(x, dtype=np.float64)
    bits = np.zeros(len(x), dtype=np.uint16)
    code = N.FE_PREC_BF16 if prec == "bf16" else N.FE_PREC_FP16
    assert N.lib.fe_round16(ctypes.c_void_p(x.ctypes.data), len(x), code,
                            ctypes.c_void_p(bits.ctypes.data)) == 0
    for xi, b in zip(x, bits):
        r = _round_ref(float(xi), p, emin, emax)
        if prec == "bf16":
            assert b == _bits_bf16(r), (xi, hex(b), r)
        else:
            assert b == int(np.array([r], dtype=np.float16).view(np.uint16)[0]), (xi, hex(b), r)
    # NaN stays NaN
    nan = np.array([np.nan], dtype=np.float64)
    assert N.lib.fe_round16(ctypes.c_void_p(nan.ctypes.data), 1, code, ctypes.c_void_p(bits.ctypes.data)) == 0
    mask = (0x7F80, 0x7F) if prec == "bf16" else (0x7C00, 0x3FF)
    assert (bits[0] & mask[0]) == mask[0] and (bits[0] & mask[1])


def test_round16_agrees_with_numpy_half(fe):
    """numpy's binary64 -> binary16 conversion is an independent implementation."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    rng = np.random.default_rng(12)
    x = rng.standard_normal(200_000) * 2.0 ** rng.integers(-30, 18, 200_000)
    bits = np.zeros(len(x), dtype=np.uint16)
    assert N.lib.fe_round16(ctypes.c_void_p(x.ctypes.data), len(x), N.FE_PREC_FP16,
                            ctypes.c_void_p(bits.ctypes.data)) == 0
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(bits, ref)
    assert N.lib.fe_round16(ctypes.c_void_p(x.ctypes.data), 1, N.FE_PREC_FP64, ctypes.c_void_p(bits.ctypes.data)) != 0


@pytest.mark.parametrize("from_binary32", [0, 1])
def test_round_tf32_matches_ieee_definition(fe, from_binary32):
    """fe_round_tf32 (the TF32 plans' rounding of tables and DoFs, and of the
    binary32 pointwise results) against round-to-nearest-even to 11 significand
    bits with binary32's exponent range, written from its definition."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    rng = np.random.default_rng(13)
    p, emin, emax = 11, -126, 127
    x = list(rng.standard_normal(3000) * 2.0 ** rng.integers(emin - 14, emax + 2, 3000))
    for _ in range(1500):
        e = int(rng.integers(emin - 8, emax))
        m = int(rng.integers(2 ** (p - 1), 2 ** p))
        t = (m + 0.5) * 2.0 ** (e - p + 1)
        x += [t, -t, np.nextafter(t, 0), np.nextafter(t, np.inf)]
    big = (2 - 2.0 ** (1 - p)) * 2.0 ** emax
    x += [0.0, -0.0, np.inf, -np.inf, big, big + 2.0 ** (emax - p), np.nextafter(big + 2.0 ** (emax - p), 0),
          2.0 ** (emin - p + 1), 2.0 ** (emin - p), np.nextafter(2.0 ** (emin - p), 1), 1e-300, 5e-324]
    x = np.asarray(x, dtype=np.float64)
    bits = np.zeros(len(x), dtype=np.uint32)
    assert N.lib.fe_round_tf32(ctypes.c_void_p(x.ctypes.data), len(x), from_binary32,
                               ctypes.c_void_p(bits.ctypes.data)) == 0
    with np.errstate(over="ignore"):
        src = x.astype(np.float32).astype(np.float64) if from_binary32 else x
    for xi, si, b in zip(x, src, bits):
        r = _round_ref(float(si), p, emin, emax)
        want = int(np.array([r], dtype=np.float32).view(np.uint32)[0])
        assert b == want, (xi, from_binary32, hex(int(b)), r)
        assert b & 0x1FFF == 0
    nan = np.array([np.nan], dtype=np.float64)
    assert N.lib.fe_round_tf32(ctypes.c_void_p(nan.ctypes.data), 1, from_binary32,
                               ctypes.c_void_p(bits.ctypes.data)) == 0
    assert (bits[0] & 0x7F800000) == 0x7F800000 and (bits[0] & 0x7FE000)


def test_round_tf32_and_round16_reject_null(fe):
    """Documented errors of the host rounding entry points."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    null = ctypes.c_void_p(0)
    assert N.lib.fe_round_tf32(null, 4, 0, null) == N.FE_ERR_INVALID_ARG
    assert N.lib.fe_round_tf32(null, 0, 1, null) == N.FE_OK          # nothing to round
    assert N.lib.fe_round16(null, 3, N.FE_PREC_BF16, null) == N.FE_ERR_INVALID_ARG
    x = np.zeros(2)
    b = np.zeros(2, dtype=np.uint16)
    assert N.lib.fe_round16(ctypes.c_void_p(x.ctypes.data), 2, N.FE_PREC_TF32,
                            ctypes.c_void_p(b.ctypes.data)) == N.FE_ERR_UNSUPPORTED


def test_plan_create_rejects_out_of_range_sizes(fe):
    """Host-side argument checks of fe_plan_create run before any device call, so
    they are testable without a GPU: DoF indices must fit int32 (n_nodes x
    components < 2^31), the quadrature degree is at most 40, the kind and the
    precision must be known.  The pointers are never dereferenced here."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    fake = ctypes.c_void_p(0x10000)   # 16-byte aligned, never touched on these paths

    def create(dim=3, degree=2, n_nodes=1000, kind=N.FE_FORM_ELASTICITY, q=2, prec=N.FE_PREC_FP64):
        mesh = N.FeMesh(dim, degree, 100, 10, n_nodes, fake, fake, fake)
        form = N.FeForm(kind, q, prec, 0, 1.25, 1.0, None, None, None, 0, 0)
        h = ctypes.c_void_p(0)
        return N.lib.fe_plan_create(ctypes.byref(form), ctypes.byref(mesh), ctypes.byref(h))

    # 3 components x 715,827,883 nodes = 2^31 + 1: too many DoFs for int32 indices
    assert create(n_nodes=715_827_883) == N.FE_ERR_INVALID_ARG
    assert create(q=41) == N.FE_ERR_INVALID_ARG
    assert create(kind=99) == N.FE_ERR_INVALID_ARG
    assert create(prec=17) == N.FE_ERR_UNSUPPORTED
    assert create(dim=4) == N.FE_ERR_INVALID_ARG
    assert create(kind=N.FE_FORM_NH_RESIDUAL, prec=N.FE_PREC_FP16) == N.FE_ERR_UNSUPPORTED


def test_noalloc_refuses_plan_options_it_cannot_honour(fe):
    """fe_action_noalloc runs only the plain thread-per-cell kernel with the atomic
    scatter.  A form asking for another plan option (node-ordered scatter,
    cells-per-CTA kernel, global tables, a block size) is refused with
    FE_ERR_UNSUPPORTED before any device call, so no caller silently gets a
    different scatter than it asked for."""
    import ctypes
    from paper_2506_17471_gb300 import _native as N
    fake = ctypes.c_void_p(0x10000)   # never dereferenced on these paths
    mesh = N.FeMesh(3, 2, 100, 10, 1000, fake, fake, fake)
    tab = np.zeros(4 * 4 * 10)
    wts = np.zeros(4)

    def call(flags=0, tile=0, prec=N.FE_PREC_FP64):
        form = N.FeForm(N.FE_FORM_ELASTICITY, 2, prec, flags, 1.25, 1.0, None, None, None, tile, 0)
        return N.lib.fe_action_noalloc(ctypes.byref(form), ctypes.byref(mesh),
                                       tab.ctypes.data_as(ctypes.c_void_p),
                                       wts.ctypes.data_as(ctypes.c_void_p), 4,
                                       fake, ctypes.c_void_p(0x20000), None, None)

    for flag in (N.FE_FLAG_GATHER_SCATTER, N.FE_FLAG_COOPERATIVE, N.FE_FLAG_TABLES_GLOBAL,
                 N.FE_FLAG_ACCUMULATE | N.FE_FLAG_GATHER_SCATTER, 1 << 7):
        assert call(flags=flag) == N.FE_ERR_UNSUPPORTED, flag
    assert call(tile=64) == N.FE_ERR_UNSUPPORTED
    assert call(prec=N.FE_PREC_FP32) == N.FE_ERR_UNSUPPORTED
