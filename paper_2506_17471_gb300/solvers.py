"""Conjugate gradients and FP64 iterative refinement around a reduced-precision action.

The operator is a plan's action (``plan.apply``); the vector work of every
iteration runs in the library's CUDA kernels (``fe_cg_*``), with all scalars on
the device, so a block of iterations is captured once in a CUDA graph and
replayed; the host reads the residual norm once per block.

Dirichlet DoFs are handled by a 0/1 mask M (1 = free): the solved system is
M A M + (I - M), right-hand sides are masked, and every CG vector stays zero on
the masked DoFs.

Iterative refinement (the FP64 refinement of the mixed-precision form): with
x_0 = 0, repeat r_k = M (b - A_64 x_k) in FP64; stop when ||r_k|| <= tol ||M b||;
otherwise solve A_low d = r_k by CG to a relative tolerance ``inner_rtol`` with
the reduced-precision action, and set x_{k+1} = x_k + d.
"""

from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import torch

from . import _native as N

S_RR, S_PQ, S_ALPHA, S_BETA, S_RRNEW, S_DOT = 0, 1, 2, 3, 4, 5


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Workspace:
    """Device vectors and the reduction workspace for one CG solve of size n."""

    def __init__(self, n: int, device):
        self.n = int(n)
        self.ws = torch.zeros(N.FE_CG_WORKSPACE_DOUBLES, dtype=torch.float64, device=device)
        self.r = torch.zeros(n, dtype=torch.float64, device=device)
        self.p = torch.zeros_like(self.r)
        self.q = torch.zeros_like(self.r)

    def scalar(self, s: int) -> float:
        return float(self.ws[N.FE_CG_PARTIALS + s].item())

    def dot(self, x, y, mask=None, slot=S_DOT) -> float:
        N.check(N.lib.fe_vec_dot(self.n, _p(x), _p(y), _p(mask), _p(self.ws), slot, _s()), "fe_vec_dot")
        return self.scalar(slot)


@dataclass
class SolveStats:
    iterations: int = 0
    outer: int = 0
    rel_residual: float = float("nan")
    history: list = field(default_factory=list)


def cg(apply, b: torch.Tensor, mask: torch.Tensor | None = None, x: torch.Tensor | None = None,
       rtol: float = 1e-10, maxiter: int = 20000, block: int = 25, use_graph: bool = True,
       work: Workspace | None = None) -> tuple[torch.Tensor, SolveStats]:
    """Solve (M A M + I - M) x = M b by CG.  ``apply(u, y)`` writes y = A u.

    Convergence is tested every ``block`` iterations on the recursively updated
    residual: ||r|| <= rtol ||M b||."""
    n = b.numel()
    w = work or Workspace(n, b.device)
    if x is None:
        x = torch.zeros_like(b)
    stats = SolveStats()
    bb = w.dot(b, b, mask)
    if bb == 0.0:
        x.zero_()
        stats.rel_residual = 0.0
        return x, stats
    target = rtol * rtol * bb
    apply(x, w.q)
    N.check(N.lib.fe_cg_start(n, _p(b), _p(w.q), _p(mask), _p(w.r), _p(w.p), _p(w.ws), _s()),
            "fe_cg_start")
    rr = w.scalar(S_RR)
    if rr <= target:
        stats.rel_residual = math.sqrt(rr / bb)
        return x, stats

    def iterations(k):
        for _ in range(k):
            apply(w.p, w.q)
            N.lib.fe_cg_direction(n, _p(w.p), _p(w.q), _p(mask), _p(w.ws), _s())
            N.lib.fe_cg_update(n, _p(x), _p(w.r), _p(w.p), _p(w.q), _p(w.ws), _s())
            N.lib.fe_cg_new_direction(n, _p(w.r), _p(w.p), _p(w.ws), _s())

    graph = None
    if use_graph:
        # capture one block of iterations; the vectors and scalars it touches are static
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            iterations(block)
        # capturing does not execute the work
    while stats.iterations < maxiter:
        if graph is not None:
            graph.replay()
        else:
            iterations(block)
        stats.iterations += block
        rr = w.scalar(S_RR)
        stats.history.append(math.sqrt(max(rr, 0.0) / bb))
        if rr <= target or not math.isfinite(rr):
            break
    stats.rel_residual = math.sqrt(max(rr, 0.0) / bb)
    return x, stats


def cg_ir(apply_hi, apply_lo, b: torch.Tensor, mask: torch.Tensor | None = None, tol: float = 1e-10,
          inner_rtol: float = 1e-5, max_outer: int = 40, block: int = 25,
          use_graph: bool = True) -> tuple[torch.Tensor, SolveStats]:
    """FP64 iterative refinement around CG with a reduced-precision action.

    Outer residuals use ``apply_hi`` (the FP64 action); each correction solves
    with ``apply_lo``.  Returns x with ||M (b - A_64 x)|| <= tol ||M b|| when it
    converges, and the per-step true relative residuals in ``history``."""
    n = b.numel()
    x = torch.zeros_like(b)
    d = torch.zeros_like(b)
    outer = Workspace(n, b.device)
    inner = Workspace(n, b.device)
    stats = SolveStats()
    bb = outer.dot(b, b, mask)
    if bb == 0.0:
        stats.rel_residual = 0.0
        return x, stats
    rvec = torch.zeros_like(b)
    for k in range(max_outer + 1):
        apply_hi(x, outer.q)
        N.check(N.lib.fe_cg_start(n, _p(b), _p(outer.q), _p(mask), _p(rvec), _p(outer.p),
                                  _p(outer.ws), _s()), "fe_cg_start")
        rel = math.sqrt(max(outer.scalar(S_RR), 0.0) / bb)
        stats.history.append(rel)
        stats.rel_residual = rel
        if rel <= tol or k == max_outer or not math.isfinite(rel):
            break
        d.zero_()
        _, st = cg(apply_lo, rvec, mask, x=d, rtol=inner_rtol, block=block, use_graph=use_graph,
                   work=inner)
        stats.iterations += st.iterations
        N.check(N.lib.fe_vec_axpy(n, 1.0, _p(d), _p(x), _s()), "fe_vec_axpy")
        stats.outer += 1
    return x, stats
