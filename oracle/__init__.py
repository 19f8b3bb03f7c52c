"""CPU FP64 oracle for the matrix-free finite element action (test infrastructure).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline (and its reference arm) may import this package.  The product package
never imports it and it never imports the product package: the two share no
code, headers, tables or helpers.

* ``quadrature.py``: conical-product Gauss-Jacobi rules (Golub-Welsch, numpy).
* ``basis.py``: Silvester-product Lagrange basis and tabulation (numpy).
* ``symmetric.py``: fully symmetric rules from the moment equations (scipy).
* ``oracle.c``: the plain cell-wise quadrature sum of every form, one cell and one
  quadrature point at a time, built with gcc into ``oracle/_build/liboracle.so``
  by :func:`build`.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (exactness, closed forms, invariants, exact rational
element matrices, finite differences).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import basis, quadrature
from .basis import tabulate

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (portable C11, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            D = ctypes.c_double
            common = [I, I, I, P, P, P, P, P]
            lib.orc_mass.argtypes = common + [P, P, L, L]
            lib.orc_elasticity.argtypes = common + [D, D, P, P, L, L]
            lib.orc_nh_residual.argtypes = common + [P, P, P, P, L, L]
            lib.orc_nh_jacobian.argtypes = common + [P, P, P, P, P, L, L]
            lib.orc_nh_energy.argtypes = common + [P, P, P, P, L, L]
            lib.orc_nh_adjoint.argtypes = common + [P, P, P, P, P, P, P, L, L]
            lib.orc_laplace.argtypes = common + [P, P, L, L]
            lib.orc_helmholtz.argtypes = common + [P, P, L, L]
            lib.orc_svk_residual.argtypes = common + [P, P, P, P, L, L]
            lib.orc_svk_jacobian.argtypes = common + [P, P, P, P, P, L, L]
            lib.orc_svk_energy.argtypes = common + [P, P, P, P, L, L]
            for f in (lib.orc_mass, lib.orc_elasticity, lib.orc_nh_residual,
                      lib.orc_nh_jacobian, lib.orc_nh_energy, lib.orc_nh_adjoint, lib.orc_laplace,
                      lib.orc_helmholtz, lib.orc_svk_residual, lib.orc_svk_jacobian, lib.orc_svk_energy):
                f.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


_ERRORS = {1: "degenerate or non-finite cell Jacobian", 2: "det F <= 0 at a quadrature point",
           3: "bad argument"}


class OracleError(RuntimeError):
    pass


class Oracle:
    """The oracle bound to one mesh, degree and quadrature degree.

    ``coords [nv, d]``, ``cell2vertex [nc, d+1]``, ``cell2node [nc, n_loc]`` follow
    the layout conventions of ``oracle.c``; ``n_nodes`` is the global node count.
    """

    def __init__(self, dim, degree, quad_degree, coords, cell2vertex, cell2node, n_nodes,
                 scheme="conical"):
        self.dim, self.degree, self.quad_degree = int(dim), int(degree), int(quad_degree)
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.c2v = np.ascontiguousarray(cell2vertex, dtype=np.int32)
        self.c2n = np.ascontiguousarray(cell2node, dtype=np.int32)
        self.n_nodes = int(n_nodes)
        self.n_cells = int(self.c2v.shape[0])
        self.pts, self.wts, tab = tabulate(self.dim, self.degree, self.quad_degree, scheme)
        self.tab = np.ascontiguousarray(tab)
        self.nloc = int(self.tab.shape[2])
        self.nq = int(self.wts.shape[0])
        assert self.c2n.shape == (self.n_cells, self.nloc)

    @classmethod
    def from_mesh(cls, mesh, quad_degree, scheme="conical"):
        return cls(mesh.dim, mesh.degree, quad_degree, mesh.coords, mesh.cell2vertex,
                   mesh.cell2node, mesh.n_nodes, scheme)

    # ------------------------------------------------------------------ driver
    def _common(self):
        return [self.dim, self.nloc, self.nq, _ptr(self.wts), _ptr(self.tab), _ptr(self.c2v),
                _ptr(self.coords), _ptr(self.c2n)]

    def _run(self, fn, make_args, outs_shapes, threads=1, cells=None):
        """Run ``fn`` over cell ranges; each thread adds into private outputs that
        are summed afterwards (ctypes releases the GIL during the C call)."""
        c0, c1 = (0, self.n_cells) if cells is None else cells
        threads = max(1, min(int(threads), c1 - c0 if c1 > c0 else 1))
        bounds = np.linspace(c0, c1, threads + 1).astype(np.int64)
        outs = [[np.zeros(s) for s in outs_shapes] for _ in range(threads)]
        codes = [0] * threads

        def work(t):
            args = make_args(outs[t]) + [int(bounds[t]), int(bounds[t + 1])]
            codes[t] = fn(*(self._common() + args))

        if threads == 1:
            work(0)
        else:
            ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
            for th in ths:
                th.start()
            for th in ths:
                th.join()
        for code in codes:
            if code:
                raise OracleError(_ERRORS.get(code, f"code {code}"))
        res = outs[0]
        for t in range(1, threads):
            for a, b in zip(res, outs[t]):
                a += b
        return res

    def _vec(self, u, nc):
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (self.n_nodes * nc,):
            raise ValueError(f"expected {self.n_nodes * nc} DoFs, got {u.shape}")
        return u

    def _cellvec(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.n_cells,):
            raise ValueError("expected one value per cell")
        return a

    # ------------------------------------------------------------------ forms
    def mass(self, u, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, 1)
        (y,) = self._run(lib.orc_mass, lambda o: [_ptr(u), _ptr(o[0])],
                         [(self.n_nodes,)], threads, cells)
        return y

    def elasticity(self, u, lam, mu, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, self.dim)
        (y,) = self._run(lib.orc_elasticity,
                         lambda o: [float(lam), float(mu), _ptr(u), _ptr(o[0])],
                         [(self.n_nodes * self.dim,)], threads, cells)
        return y

    def nh_residual(self, u, mu_cell, lam_cell, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (y,) = self._run(lib.orc_nh_residual,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(o[0])],
                         [(self.n_nodes * self.dim,)], threads, cells)
        return y

    def nh_jacobian(self, u, du, mu_cell, lam_cell, threads=1, cells=None):
        lib = _load()
        u, du = self._vec(u, self.dim), self._vec(du, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (y,) = self._run(lib.orc_nh_jacobian,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(du), _ptr(o[0])],
                         [(self.n_nodes * self.dim,)], threads, cells)
        return y

    def nh_energy(self, u, mu_cell, lam_cell, threads=1):
        """Per-cell energies; their sum is Pi(u)."""
        lib = _load()
        u = self._vec(u, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (e,) = self._run(lib.orc_nh_energy,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(o[0])],
                         [(self.n_cells,)], threads)
        return e

    def nh_adjoint(self, u, w, mu_cell, lam_cell, threads=1, cells=None):
        """(J(u)^T w, dmu [n_cells], dlambda [n_cells])."""
        lib = _load()
        u, w = self._vec(u, self.dim), self._vec(w, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        jtw, dmu, dlam = self._run(
            lib.orc_nh_adjoint,
            lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(w), _ptr(o[0]), _ptr(o[1]), _ptr(o[2])],
            [(self.n_nodes * self.dim,), (self.n_cells,), (self.n_cells,)], threads, cells)
        return jtw, dmu, dlam

    def laplace(self, u, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, 1)
        (y,) = self._run(lib.orc_laplace, lambda o: [_ptr(u), _ptr(o[0])],
                         [(self.n_nodes,)], threads, cells)
        return y

    def helmholtz(self, u, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, 1)
        (y,) = self._run(lib.orc_helmholtz, lambda o: [_ptr(u), _ptr(o[0])],
                         [(self.n_nodes,)], threads, cells)
        return y

    def svk_residual(self, u, mu_cell, lam_cell, threads=1, cells=None):
        lib = _load()
        u = self._vec(u, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (y,) = self._run(lib.orc_svk_residual,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(o[0])],
                         [(self.n_nodes * self.dim,)], threads, cells)
        return y

    def svk_jacobian(self, u, du, mu_cell, lam_cell, threads=1, cells=None):
        lib = _load()
        u, du = self._vec(u, self.dim), self._vec(du, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (y,) = self._run(lib.orc_svk_jacobian,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(du), _ptr(o[0])],
                         [(self.n_nodes * self.dim,)], threads, cells)
        return y

    def svk_energy(self, u, mu_cell, lam_cell, threads=1):
        """Per-cell St. Venant-Kirchhoff energies; their sum is Pi(u)."""
        lib = _load()
        u = self._vec(u, self.dim)
        mu, lam = self._cellvec(mu_cell), self._cellvec(lam_cell)
        (e,) = self._run(lib.orc_svk_energy,
                         lambda o: [_ptr(mu), _ptr(lam), _ptr(u), _ptr(o[0])],
                         [(self.n_cells,)], threads)
        return e

    # ------------------------------------------------------------------ dense
    def dense(self, apply, n):
        """Dense matrix with columns apply(e_j), j < n (tiny meshes only)."""
        A = np.empty((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[j] = 1.0
            A[:, j] = apply(e)
            e[j] = 0.0
        return A


__all__ = ["Oracle", "OracleError", "build", "tabulate", "basis", "quadrature"]
