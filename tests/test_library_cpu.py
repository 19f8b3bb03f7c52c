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


@pytest.mark.parametrize("dim,q", [(2, 2), (2, 4), (2, 6), (2, 8), (3, 2), (3, 4), (3, 5), (3, 6)])
@pytest.mark.parametrize("degree", [1, 2, 4])
def test_symmetric_tabulation_matches_oracle(fe, dim, q, degree):
    import oracle
    pts, wts, tab = fe.tabulate(dim, degree, q, "symmetric")
    p2, w2, t2 = oracle.tabulate(dim, degree, q, "symmetric")
    if (dim, q) in ((3, 6),):   # no tabulated symmetric rule: the conical-product fallback
        np.testing.assert_allclose(pts, p2, rtol=0, atol=1e-15)
        np.testing.assert_allclose(wts, w2, rtol=1e-14)
    else:                        # both sides round the extended-precision solution once
        assert np.array_equal(pts, p2) and np.array_equal(wts, w2)
    assert np.abs(tab - t2).max() <= 1e-14 * np.abs(t2).max()
