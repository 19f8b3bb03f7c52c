"""Conditioning of the FP64 evaluation on the full-size Neo-Hookean workload (no GPU).

Two correct FP64 implementations whose tabulations differ only in the last bit
cannot agree better than the problem's conditioning allows.  On the 256^2 P4
mesh with the smooth 8-mode sinusoid displacement, the residual is evaluated
from displacement gradients that are sums of nodal terms about 1e3 times larger
than the result; this test measures the oracle's own sensitivity to a random
half-ulp perturbation of its tabulation, which justifies the residual's parity
tolerance of 1e-11 (about 7x the measured sensitivity) while the Jacobian action
along a rough direction stays within 1e-12.
"""

import numpy as np

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.fields import sinusoid_displacement


def test_nh_residual_smooth_field_sensitivity(oracle_built):
    m = structured_mesh(2, 256, 4, jitter=0.2, seed=20250619)
    o = oracle.Oracle.from_mesh(m, 8)
    mu, lam = lame_fields(m.n_cells, 3)
    u = sinusoid_displacement(m, 4)
    r = o.nh_residual(u, mu, lam, threads=8)
    w = uniform_field(m.n_nodes * 2, 5)
    j = o.nh_jacobian(u, w, mu, lam, threads=8)
    cells = (0, 1500)
    _, dmu, _ = o.nh_adjoint(u, w, mu, lam, threads=8, cells=cells)
    rng = np.random.default_rng(0)
    t0 = o.tab.copy()
    o.tab = np.ascontiguousarray(t0 * (1 + 2.0 ** -53 * rng.choice([-1.0, 1.0], size=t0.shape)))
    dr = np.abs(o.nh_residual(u, mu, lam, threads=8) - r).max() / np.abs(r).max()
    dj = np.abs(o.nh_jacobian(u, w, mu, lam, threads=8) - j).max() / np.abs(j).max()
    _, dmu2, _ = o.nh_adjoint(u, w, mu, lam, threads=8, cells=cells)
    ddmu = np.abs(dmu2 - dmu)[:1500].max() / np.abs(dmu[:1500]).max()
    assert 5e-13 < dr < 5e-12, dr      # residual: rounding alone reaches ~1.5e-12
    assert dj < 5e-13, dj              # rough-direction Jacobian: well conditioned
    assert ddmu < 2e-12, ddmu          # dmu uses the same smooth-field gradients
    print(f"sensitivity: residual {dr:.2e}, jacobian {dj:.2e}, dmu {ddmu:.2e}")


def test_nh_jacobian_p6_smooth_linearisation_sensitivity(oracle_built):
    """hp-sweep Neo-Hookean Jacobian (P6 triangles, 236^2 x 2 cells): linearised at
    the smooth sinusoid field, a half-ulp tabulation change moves the oracle's own
    result by ~5e-13, so an independent FP64 evaluation differing in operation
    order lands at ~1e-12; the parity tolerance there is 1e-11."""
    m = structured_mesh(2, 236, 6, jitter=0.2, seed=20250620 + 236)
    o = oracle.Oracle.from_mesh(m, 12)
    mu, lam = lame_fields(m.n_cells, 2)
    ul = sinusoid_displacement(m, 3)
    du = uniform_field(m.n_nodes * 2, 4)
    j = o.nh_jacobian(ul, du, mu, lam, threads=8)
    rng = np.random.default_rng(0)
    t0 = o.tab.copy()
    o.tab = np.ascontiguousarray(t0 * (1 + 2.0 ** -53 * rng.choice([-1.0, 1.0], size=t0.shape)))
    dj = np.abs(o.nh_jacobian(ul, du, mu, lam, threads=8) - j).max() / np.abs(j).max()
    assert 1e-13 < dj < 5e-12, dj
