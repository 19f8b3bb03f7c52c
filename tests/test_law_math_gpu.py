"""The Neo-Hookean laws' logarithm and reciprocal on the GPU (fe_selftest_log_rcp).

The kernels evaluate log det F by Tang's table-driven method and 1/det F by the
approximate hardware reciprocal refined by two Newton-Raphson steps instead of
CUDA's log and the IEEE division (fewer FP64 instructions per quadrature point).
Both are held to CUDA's documented bound for log (1 ulp; the division is
correctly rounded, 0.5 ulp, so the reciprocal is held to 1 ulp too) against a
reference in numpy's long double (IEEE quadruple precision on the aarch64 host
of the GPU, 80-bit extended on x86), over arguments spread across the whole
normal range, clustered around 1 (where det F lies), at the table's interval
ends and at the square-root-of-two split.  Arguments outside the normal range
take CUDA's log and the IEEE division, and must match them exactly.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2506_17471_gb300 import _native
    return _native


def run(N, x):
    xd = torch.from_numpy(x).cuda()
    lo, rc = torch.empty_like(xd), torch.empty_like(xd)
    tab = torch.empty(N.FE_LOG_TABLE_DOUBLES, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    assert N.lib.fe_selftest_log_rcp(P(xd.data_ptr()), len(x), P(tab.data_ptr()), P(lo.data_ptr()),
                                     P(rc.data_ptr()), s) == 0
    torch.cuda.synchronize()
    return lo.cpu().numpy(), rc.cpu().numpy(), xd


def arguments():
    rng = np.random.default_rng(7)
    parts = [
        np.exp(rng.uniform(np.log(2.0 ** -1021), np.log(2.0 ** 1023), 200_000)),   # whole normal range
        1.0 + rng.uniform(-0.5, 0.5, 200_000),                                     # det F
        1.0 + rng.uniform(-1e-6, 1e-6, 50_000),                                    # near 1
        rng.uniform(0.18, 4.0, 200_000),
    ]
    edges = []
    for i in range(90, 183):           # table points and the midpoints between them
        for k in (-3, 0, 3):
            c = i / 128.0
            edges += [np.nextafter(c, 0) if k < 0 else c, c + (0.5 / 128.0), c - (0.5 / 128.0)]
    s2 = np.sqrt(2.0)
    edges += [s2, np.nextafter(s2, 0), np.nextafter(s2, 2), s2 / 2, np.nextafter(s2 / 2, 0), 1.0,
              np.nextafter(1.0, 0), np.nextafter(1.0, 2), 2.0, 0.5, 2.0 ** -1022, np.finfo(float).max]
    e = np.array(edges, dtype=np.float64)
    scaled = np.concatenate([e * 2.0 ** k for k in (-600, -7, 0, 9, 500)])
    x = np.concatenate(parts + [e, scaled])
    return x[np.isfinite(x) & (x >= 2.0 ** -1022)]


def ulp_err(got, ref_ld):
    ref = ref_ld.astype(np.float64)
    sp = np.spacing(np.abs(ref))
    return np.abs((got.astype(np.longdouble) - ref_ld) / sp.astype(np.longdouble)).astype(np.float64)


def test_log_and_reciprocal_within_one_ulp(N):
    x = arguments()
    lo, rc, xd = run(N, x)
    xl = x.astype(np.longdouble)
    err_log = ulp_err(lo, np.log(xl))
    err_rcp = ulp_err(rc, np.longdouble(1) / xl)
    # CUDA's own log measured the same way, for comparison
    err_cuda = ulp_err(torch.log(xd).cpu().numpy(), np.log(xl))
    print(f"max ulp: table log {err_log.max():.3f}, CUDA log {err_cuda.max():.3f}, "
          f"reciprocal {err_rcp.max():.3f}")
    assert err_log.max() <= 1.0
    assert err_rcp.max() <= 1.0
    assert np.all(lo[x == 1.0] == 0.0)


def test_outside_the_normal_range_defers_to_cuda(N):
    x = np.array([0.0, -0.0, -1.0, 2.0 ** -1060, 5e-324, np.inf, np.nan, -np.inf], dtype=np.float64)
    lo, rc, xd = run(N, x)
    ref_log = torch.log(xd).cpu().numpy()
    ref_rcp = (1.0 / xd).cpu().numpy()
    np.testing.assert_array_equal(lo, ref_log)
    np.testing.assert_array_equal(rc, ref_rcp)
