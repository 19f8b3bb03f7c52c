"""Python surface of the action library (argument marshalling over the C-ABI).

PyTorch provides device memory and streams; every arithmetic step of the action
runs in the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

MASS = N.FE_FORM_MASS
ELASTICITY = N.FE_FORM_ELASTICITY
NH_RESIDUAL = N.FE_FORM_NH_RESIDUAL
NH_JACOBIAN = N.FE_FORM_NH_JACOBIAN
LAPLACE = N.FE_FORM_LAPLACE
HELMHOLTZ = N.FE_FORM_HELMHOLTZ
SVK_RESIDUAL = N.FE_FORM_SVK_RESIDUAL
SVK_JACOBIAN = N.FE_FORM_SVK_JACOBIAN
FORM_NAMES = {MASS: "mass", ELASTICITY: "elasticity", NH_RESIDUAL: "nh_residual",
              NH_JACOBIAN: "nh_jacobian", LAPLACE: "laplace", HELMHOLTZ: "helmholtz",
              SVK_RESIDUAL: "svk_residual", SVK_JACOBIAN: "svk_jacobian"}
SCALAR_FORMS = (MASS, LAPLACE, HELMHOLTZ)
# contraction precision of a plan (include/feaction.h, enum fe_precision)
PRECISIONS = {"fp64": N.FE_PREC_FP64, "fp32": N.FE_PREC_FP32, "bf16": N.FE_PREC_BF16,
              "fp16": N.FE_PREC_FP16, "fp16x2": N.FE_PREC_FP16X2, "tf32": N.FE_PREC_TF32}


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


QUAD_SCHEMES = {"conical": N.FE_QUAD_CONICAL, "symmetric": N.FE_QUAD_SYMMETRIC}


def tabulate(dim: int, degree: int, quad_degree: int, scheme: str = "conical"):
    """Quadrature points [nq,d], weights [nq], tabulation [1+d, nq, n_loc] (host)."""
    sc = QUAD_SCHEMES[scheme]
    nq = ctypes.c_int(0)
    N.check(N.lib.fe_tabulate_scheme(dim, degree, quad_degree, sc, ctypes.byref(nq), None, None, None, 0),
            "fe_tabulate")
    from math import comb
    n = comb(degree + dim, dim)
    pts = np.zeros((nq.value, dim))
    wts = np.zeros(nq.value)
    tab = np.zeros((1 + dim, nq.value, n))
    N.check(N.lib.fe_tabulate_scheme(dim, degree, quad_degree, sc, ctypes.byref(nq),
                                     pts.ctypes.data_as(ctypes.c_void_p),
                                     wts.ctypes.data_as(ctypes.c_void_p),
                                     tab.ctypes.data_as(ctypes.c_void_p), tab.size), "fe_tabulate")
    return pts, wts, tab


class Mesh:
    """Device-resident affine simplex mesh with P_degree DoF numbering.

    coords [n_vertices, dim] float64, cell2vertex [n_cells, dim+1] int32,
    cell2node [n_cells, C(degree+dim, dim)] int32 (local node order as in
    include/feaction.h)."""

    def __init__(self, dim, degree, coords, cell2vertex, cell2node, n_nodes, device="cuda"):
        self.dim, self.degree, self.n_nodes = int(dim), int(degree), int(n_nodes)
        self.coords = torch.as_tensor(np.asarray(coords), dtype=torch.float64).to(device).contiguous()
        self.cell2vertex = torch.as_tensor(np.asarray(cell2vertex), dtype=torch.int32).to(device).contiguous()
        self.cell2node = torch.as_tensor(np.asarray(cell2node), dtype=torch.int32).to(device).contiguous()
        self.device = self.coords.device

    @property
    def n_cells(self) -> int:
        return int(self.cell2vertex.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    def _c(self) -> N.FeMesh:
        return N.FeMesh(self.dim, self.degree, self.n_vertices, self.n_cells, self.n_nodes,
                        self.coords.data_ptr(), self.cell2vertex.data_ptr(),
                        self.cell2node.data_ptr())


@dataclass
class PlanInfo:
    nq: int
    n_loc: int
    ncomp: int
    kernel: int
    threads_per_block: int
    grid_blocks: int
    n_dofs: int
    flops_per_cell: float
    bytes_min: float
    flops_per_cell_dense: float


class Plan:
    """A form bound to a mesh: tables uploaded once, kernel selected once.

    kind: MASS, ELASTICITY, NH_RESIDUAL, NH_JACOBIAN, LAPLACE, HELMHOLTZ, SVK_RESIDUAL
    or SVK_JACOBIAN.  Hyperelastic (Neo-Hookean, St. Venant-Kirchhoff) kinds take
    per-cell ``mu_cell``/``lam_cell`` (copied into plan-owned device buffers that
    :meth:`set_lame` can overwrite) or the constants ``mu``/``lam``; NH_JACOBIAN
    takes the linearisation point ``u_lin`` (plan-owned copy, see
    :meth:`set_linearisation`)."""

    def __init__(self, mesh: Mesh, kind: int, quad_degree: int, *, lam: float = 0.0,
                 mu: float = 0.0, mu_cell=None, lam_cell=None, u_lin=None,
                 accumulate: bool = False, precision: str = "fp64", cooperative: bool = False,
                 tile_cells: int = 0, tables_global: bool = False, quad_scheme: str = "conical",
                 gather_scatter: bool = False):
        self.mesh = mesh
        self.kind = int(kind)
        self.ncomp = 1 if kind in SCALAR_FORMS else mesh.dim
        dev = mesh.device
        self.mu_cell = None if mu_cell is None else torch.as_tensor(
            mu_cell, dtype=torch.float64, device=dev).clone().contiguous()
        self.lam_cell = None if lam_cell is None else torch.as_tensor(
            lam_cell, dtype=torch.float64, device=dev).clone().contiguous()
        self.u_lin = None if u_lin is None else torch.as_tensor(
            u_lin, dtype=torch.float64, device=dev).clone().contiguous()
        flags = ((N.FE_FLAG_ACCUMULATE if accumulate else 0) | (N.FE_FLAG_COOPERATIVE if cooperative else 0)
                 | (N.FE_FLAG_TABLES_GLOBAL if tables_global else 0)
                 | (N.FE_FLAG_GATHER_SCATTER if gather_scatter else 0))
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.precision = precision
        self._form = N.FeForm(self.kind, int(quad_degree), PRECISIONS[precision], flags, float(lam),
                              float(mu), _dptr(self.lam_cell).value or 0,
                              _dptr(self.mu_cell).value or 0, _dptr(self.u_lin).value or 0,
                              int(tile_cells), QUAD_SCHEMES[quad_scheme])
        self._mesh_c = mesh._c()
        handle = ctypes.c_void_p(0)
        N.check(N.lib.fe_plan_create(ctypes.byref(self._form), ctypes.byref(self._mesh_c),
                                     ctypes.byref(handle)), "fe_plan_create")
        self._h = handle
        info = N.FePlanInfo()
        N.check(N.lib.fe_plan_get_info(self._h, ctypes.byref(info)), "fe_plan_get_info")
        self.info = PlanInfo(info.nq, info.n_loc, info.ncomp, info.kernel, info.threads_per_block,
                             info.grid_blocks, info.n_dofs, info.flops_per_cell, info.bytes_min,
                             info.flops_per_cell_dense)

    @property
    def n_dofs(self) -> int:
        return self.mesh.n_nodes * self.ncomp

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib.fe_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self) -> "Plan":
        return self

    def __exit__(self, *exc) -> None:
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_lame(self, mu_cell=None, lam_cell=None):
        if mu_cell is not None:
            self.mu_cell.copy_(torch.as_tensor(mu_cell, dtype=torch.float64))
        if lam_cell is not None:
            self.lam_cell.copy_(torch.as_tensor(lam_cell, dtype=torch.float64))

    def set_linearisation(self, u_lin):
        self.u_lin.copy_(torch.as_tensor(u_lin, dtype=torch.float64))

    def _check_vec(self, t: torch.Tensor, name: str):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n_dofs:
            raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor of {self.n_dofs} values")

    def apply(self, u: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = A(u) on the current (or given) stream; asynchronous.

        A host (CPU) ``u`` is copied to the device and the result copied back."""
        if not u.is_cuda:
            return self.apply_host(u)
        self._check_vec(u, "u")
        if y is None:
            y = torch.empty_like(u)
        self._check_vec(y, "y")
        N.check(N.lib.fe_action(self._h, _dptr(u), _dptr(y), _stream_ptr(stream)), "fe_action")
        return y

    def apply_host(self, u_host: torch.Tensor, y_host: torch.Tensor | None = None,
                   u_dev: torch.Tensor | None = None, y_dev: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """End to end through ``fe_action_host``: host u -> device -> action -> host y."""
        u_host = u_host.contiguous()
        if y_host is None:
            y_host = torch.empty_like(u_host)
        dev = self.mesh.device
        u_dev = torch.empty(self.n_dofs, dtype=torch.float64, device=dev) if u_dev is None else u_dev
        y_dev = torch.empty(self.n_dofs, dtype=torch.float64, device=dev) if y_dev is None else y_dev
        N.check(N.lib.fe_action_host(self._h, _dptr(u_host), _dptr(y_host), _dptr(u_dev),
                                     _dptr(y_dev), _stream_ptr(stream)), "fe_action_host")
        return y_host

    def apply_host_pipelined(self, u_hosts, y_hosts=None, stream=None):
        """End to end over several host inputs through ``fe_action_host_pipelined``:
        copies in, actions and copies out overlap across steps (two device buffer
        pairs).  Returns the list of host results."""
        u_hosts = [u.contiguous() for u in u_hosts]
        if y_hosts is None:
            y_hosts = [torch.empty_like(u) for u in u_hosts]
        for t in list(u_hosts) + list(y_hosts):
            if t.is_cuda or t.dtype != torch.float64 or t.numel() != self.n_dofs:
                raise ValueError(f"expected host float64 tensors of {self.n_dofs} values")
        dev = self.mesh.device
        if getattr(self, "_pipe_bufs", None) is None:
            self._pipe_bufs = [torch.empty(self.n_dofs, dtype=torch.float64, device=dev) for _ in range(4)]
        ub, yb = self._pipe_bufs[:2], self._pipe_bufs[2:]
        n = len(u_hosts)
        P = ctypes.c_void_p
        up = (P * n)(*[t.data_ptr() for t in u_hosts])
        yp = (P * n)(*[t.data_ptr() for t in y_hosts])
        ud = (P * 2)(*[t.data_ptr() for t in ub])
        yd = (P * 2)(*[t.data_ptr() for t in yb])
        N.check(N.lib.fe_action_host_pipelined(self._h, n, up, yp, ud, yd, _stream_ptr(stream)),
                "fe_action_host_pipelined")
        return y_hosts

    def adjoint(self, u: torch.Tensor, w: torch.Tensor, stream=None):
        """(J(u)^T w, dmu [n_cells], dlambda [n_cells]) of the Neo-Hookean residual."""
        self._check_vec(u, "u")
        self._check_vec(w, "w")
        jtw = torch.empty_like(w)
        dmu = torch.empty(self.mesh.n_cells, dtype=torch.float64, device=w.device)
        dlam = torch.empty_like(dmu)
        N.check(N.lib.fe_action_adjoint(self._h, _dptr(u), _dptr(w), _dptr(jtw), _dptr(dmu),
                                        _dptr(dlam), _stream_ptr(stream)), "fe_action_adjoint")
        return jtw, dmu, dlam

    def status(self) -> int:
        """Read and clear the device status word (synchronises)."""
        st = ctypes.c_int(0)
        N.check(N.lib.fe_plan_status(self._h, ctypes.byref(st)), "fe_plan_status")
        return st.value

    def flops(self) -> float:
        return self.info.flops_per_cell * self.mesh.n_cells


_FIELD_KW = ("mu_cell", "lam_cell", "u_lin")


def action(mesh: Mesh, kind: int, u: torch.Tensor, quad_degree: int, y: torch.Tensor | None = None,
           *, stream=None, **plan_kw) -> torch.Tensor:
    """One-call y = A(u) (the action of Algorithm 2 for form ``kind`` on ``mesh``).

    The plan for (kind, quad_degree, options) is built on first use and kept on the
    mesh, so repeated calls pay only the kernel launch.  ``plan_kw`` are
    :class:`Plan`'s keyword options; the per-call fields ``mu_cell``, ``lam_cell``
    and ``u_lin`` are copied into the cached plan's buffers on every call that
    passes them.  A host ``u`` is copied to the device and the result back."""
    fields = {k: plan_kw.pop(k) for k in _FIELD_KW if plan_kw.get(k) is not None}
    plan_kw = {k: v for k, v in plan_kw.items() if k not in _FIELD_KW}
    key = (int(kind), int(quad_degree), tuple(sorted(plan_kw.items())), tuple(sorted(fields)))
    cache = mesh.__dict__.setdefault("_action_plans", {})
    plan = cache.get(key)
    if plan is None:
        plan = cache[key] = Plan(mesh, kind, quad_degree, **fields, **plan_kw)
    else:
        if "mu_cell" in fields or "lam_cell" in fields:
            plan.set_lame(fields.get("mu_cell"), fields.get("lam_cell"))
        if "u_lin" in fields:
            plan.set_linearisation(fields["u_lin"])
    if not u.is_cuda:
        return plan.apply_host(u, y)
    return plan.apply(u, y, stream)


def measure_fp64_peak() -> float:
    """FP64 FMA throughput of the current device in GFLOP/s (FMA = 2 flops)."""
    scratch = torch.empty(152 * 8 * 256 * 4, dtype=torch.float64, device="cuda")
    g = ctypes.c_double(0.0)
    N.check(N.lib.fe_measure_fp64_peak(_dptr(scratch), scratch.numel(), ctypes.byref(g)),
            "fe_measure_fp64_peak")
    return g.value


class NeoHookeanResidual(torch.autograd.Function):
    """r = R(u; mu, lambda) with a hand-written adjoint.

    forward runs the residual kernel; backward(w) runs the adjoint kernel, which
    recomputes the quadrature-point deformation gradients from u (nothing is
    stored between the two calls) and returns J(u)^T w, dR/dmu^T w and
    dR/dlambda^T w.  The plan's Lame buffers are shared by every call on it, so
    forward saves the fields it was given and backward writes them back before
    the adjoint: a later forward on the same plan with other fields does not
    change this call's gradients."""

    @staticmethod
    def forward(ctx, u, mu_cell, lam_cell, plan: Plan):
        if plan.kind != NH_RESIDUAL or plan.mu_cell is None or plan.lam_cell is None:
            raise ValueError("plan must be an NH_RESIDUAL plan with per-cell Lame parameters")
        mu_d = mu_cell.detach().to(torch.float64).contiguous()
        lam_d = lam_cell.detach().to(torch.float64).contiguous()
        plan.set_lame(mu_d, lam_d)
        u = u.detach().contiguous()
        ctx.save_for_backward(u, mu_d, lam_d)
        ctx.plan = plan
        return plan.apply(u)

    @staticmethod
    def backward(ctx, w):
        u, mu_d, lam_d = ctx.saved_tensors
        ctx.plan.set_lame(mu_d, lam_d)
        jtw, dmu, dlam = ctx.plan.adjoint(u, w.contiguous())
        return jtw, dmu, dlam, None


class Batch:
    """Many independent problems in one persistent launch (``fe_batch_*``).

    ``problems``: list of dicts with keys mesh (Mesh), kind (MASS, ELASTICITY or
    NH_RESIDUAL), quad_degree, u (device tensor), optional lam, mu, mu_cell,
    lam_cell, kernel (-1 auto, 0 thread-per-cell, 1 cells-per-CTA) and
    tile_cells.  Outputs are allocated here (``self.y[i]``)."""

    def __init__(self, problems):
        self._keep = []
        self.y = []
        arr = (N.FeBatchProblem * len(problems))()
        for i, pb in enumerate(problems):
            mesh = pb["mesh"]
            kind = int(pb["kind"])
            nc = 1 if kind in SCALAR_FORMS else mesh.dim
            u = pb["u"]
            if u.dtype != torch.float64 or not u.is_cuda or u.numel() != mesh.n_nodes * nc:
                raise ValueError(f"problem {i}: u must be a float64 CUDA tensor of {mesh.n_nodes * nc}")
            y = torch.empty_like(u)
            mu_cell = pb.get("mu_cell")
            lam_cell = pb.get("lam_cell")
            mu_cell = None if mu_cell is None else torch.as_tensor(mu_cell, dtype=torch.float64,
                                                                   device=u.device).contiguous()
            lam_cell = None if lam_cell is None else torch.as_tensor(lam_cell, dtype=torch.float64,
                                                                     device=u.device).contiguous()
            self._keep += [mesh, u, y, mu_cell, lam_cell]
            self.y.append(y)
            flags = N.FE_FLAG_TABLES_GLOBAL if pb.get("tables_global") else 0
            arr[i].form = N.FeForm(kind, int(pb["quad_degree"]), N.FE_PREC_FP64, flags,
                                   float(pb.get("lam", 0.0)), float(pb.get("mu", 0.0)),
                                   _dptr(lam_cell).value or 0, _dptr(mu_cell).value or 0, 0, 0,
                                   QUAD_SCHEMES[pb.get("quad_scheme", "conical")])
            arr[i].mesh = mesh._c()
            arr[i].u = u.data_ptr()
            arr[i].y = y.data_ptr()
            arr[i].kernel = int(pb.get("kernel", -1))
            arr[i].tile_cells = int(pb.get("tile_cells", 0))
        self._arr = arr
        h = ctypes.c_void_p(0)
        N.check(N.lib.fe_batch_create(arr, len(problems), ctypes.byref(h)), "fe_batch_create")
        self._h = h
        info = N.FeBatchInfo()
        N.check(N.lib.fe_batch_get_info(self._h, ctypes.byref(info)), "fe_batch_get_info")
        self.info = {"problems": info.problems, "items": info.items, "grid_blocks": info.grid_blocks,
                     "smem_bytes": info.smem_bytes, "dofs": info.dofs,
                     "contraction_flops": info.contraction_flops}

    def run(self, stream=None):
        N.check(N.lib.fe_batch_run(self._h, _stream_ptr(stream)), "fe_batch_run")
        return self.y

    def status(self) -> int:
        st = ctypes.c_int(0)
        N.check(N.lib.fe_batch_status(self._h, ctypes.byref(st)), "fe_batch_status")
        return st.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib.fe_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self) -> "Batch":
        return self

    def __exit__(self, *exc) -> None:
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
