"""Autotuner for the action's launch configuration, one problem at a time.

It follows the paper's tuning procedure (Sec. "Parameter Search Space",
"Cost Model", "Summary"): enumerate a bounded candidate space, prune it with
efficiency thresholds, rank the survivors with a heuristic cost model, time the
best ``b`` candidates on the problem's own inputs and keep the fastest.  The
parameters are this part's: the kernel (thread-per-cell, or cells-per-CTA with
a tile of C cells per CTA batch).

Candidate space (constraint 1 of the paper: tile sizes ceil(C_max / k)):
thread-per-cell when compiled for the degree, and cells-per-CTA with
C in {C_max, ceil(C_max/2), ceil(C_max/3), ...} where C_max is the largest tile
whose shared-memory plan fits the per-CTA budget.

Pruning: the cells-per-CTA kernel maps (cell, quadrature point) items and then
(cell, node) items onto 256 threads; their SIMD efficiencies are
    eta_B = C Q / (256 ceil(C Q / 256)),   eta_C = C n / (256 ceil(C n / 256))
(the paper's eta_simd applied to each phase).  Phase B carries most of the
flops, and idle lanes of one CTA are filled by the other CTA resident on the SM
(the FP64 pipe is shared per SM), so a tile is kept when eta_B >= ``eta_min``;
the largest tile is always kept.

Cost model: on GB300 the FP64 pipe, not memory, binds (machine balance 0.18
flop/B), so the paper's global + local memory time t_heur is extended with an
FP64 term and kept as the memory bound:
    t = max(flops / (F_peak eta), bytes / beta_HBM) + t_launch + rounds x t_round
where eta combines how well the launch fills the machine (and its last round,
the tail) with the lane efficiency of the cells-per-CTA phases (evaluation and
quadrature carry equal contraction flops; co-resident CTAs fill idle lanes);
see :func:`model_time`.  ``spearman`` measures how well the model ranks measured candidates
(the paper's Eq. "spearmann_rho").
"""

from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import dataclass

from . import _native as N

F_PEAK_GFLOPS = 1250.0        # FP64, from unit counts and clocks
HBM_GBS = 6790.0              # measured copy bandwidth of the GB300s
N_SMS = 152
T_LAUNCH_S = 4e-6
T_BATCH_S = 1.5e-6
COOP_BLOCK = 256
SMEM_BUDGET = 100 * 1024
SMEM_TABLE_MAX = 96 * 1024    # the library keeps larger tables in global memory


@dataclass(frozen=True)
class Candidate:
    kernel: int                  # 0 thread-per-cell, 1 cells-per-CTA
    tile_cells: int = 0          # cells per CTA batch (cells-per-CTA only)
    tables_global: bool = False  # cells-per-CTA: tables in global memory instead of shared

    def label(self) -> str:
        if self.kernel == 0:
            return "tpc"
        return f"coop{self.tile_cells}" + ("g" if self.tables_global else "")





def _coop_total_bytes(n, nq, dim, ncomp, C, fields, esz=8, tables_global=None):
    """Shared memory of the cells-per-CTA plan (mirrors the kernel's layout)."""
    if tables_global is None:
        tables_global = nq * (1 + dim) * n * esz > SMEM_TABLE_MAX
    rs = ((1 + dim) * n) | 1
    ls = (fields * n * ncomp) | 1
    es = max(dim * ncomp, 1 + dim) | 1   # gradient terms, or value + gradient
    ecs = (nq * es) | 1                  # per-cell stride of e, odd
    tab = 0 if tables_global else nq * rs * esz
    woff = (tab + 7) & ~7
    block = (woff + nq * 8 + nq * esz + 15) & ~15
    off_e = (block + C * ls * 8 + 15) & ~15
    off_nodes = (off_e + C * ecs * esz + 15) & ~15
    off_geo = (off_nodes + C * n * 4 + 15) & ~15
    # geometry records of 17 doubles, adjoint accumulators, then the node order (n ints)
    return (off_geo + C * 17 * 8 + C * 2 * 8 + n * 4 + 15) & ~15


def eta_simd(items: int, threads: int = COOP_BLOCK) -> float:
    """Fraction of useful lanes when ``items`` are spread over ``threads``."""
    if items <= 0:
        return 0.0
    return items / (threads * math.ceil(items / threads))


# highest degree with a thread-per-cell variant, per (form, dimension)
_TPC_MAX_DEGREE = {
    (N.FE_FORM_MASS, 2): 6, (N.FE_FORM_MASS, 3): 4,
    (N.FE_FORM_ELASTICITY, 2): 4, (N.FE_FORM_ELASTICITY, 3): 2,
    (N.FE_FORM_NH_RESIDUAL, 2): 4, (N.FE_FORM_NH_RESIDUAL, 3): 2,
    (N.FE_FORM_NH_JACOBIAN, 2): 4, (N.FE_FORM_NH_JACOBIAN, 3): 2,
    (N.FE_FORM_LAPLACE, 2): 4, (N.FE_FORM_LAPLACE, 3): 2,
    (N.FE_FORM_HELMHOLTZ, 2): 4, (N.FE_FORM_HELMHOLTZ, 3): 2,
    (N.FE_FORM_SVK_RESIDUAL, 2): 3, (N.FE_FORM_SVK_RESIDUAL, 3): 2,
    (N.FE_FORM_SVK_JACOBIAN, 2): 3, (N.FE_FORM_SVK_JACOBIAN, 3): 1,
}


def tpc_available(kind: int, dim: int, degree: int) -> bool:
    return 1 <= degree <= _TPC_MAX_DEGREE.get((kind, dim), 0)


def candidates(kind, dim, degree, nq, n_loc, ncomp, fields=1, eta_min=0.3, max_tiles=6):
    out = []
    if tpc_available(kind, dim, degree):
        out.append(Candidate(0))
    # table residency: shared memory when the table fits, always also global memory
    residencies = [True]
    if nq * (1 + dim) * n_loc * 8 <= SMEM_TABLE_MAX:
        residencies.insert(0, False)
    for gt in residencies:
        cmax = 1
        for C in range(1, 65):
            if _coop_total_bytes(n_loc, nq, dim, ncomp, C, fields, tables_global=gt) <= SMEM_BUDGET:
                cmax = C
        seen = set()
        for k in range(1, 64):
            C = math.ceil(cmax / k)
            if C in seen:
                continue
            seen.add(C)
            if C == cmax or eta_simd(C * nq) >= eta_min:
                out.append(Candidate(1, C, gt))
            if len(seen) >= max_tiles or C == 1:
                break
    return out


SMEM_PER_SM = 228 * 1024
TAIL_GATHER = 0.05            # a tail item's gather phase, as a fraction of a whole unit
WARPS_TO_FILL_SM = 8          # warps per SM that keep the FP64 pipe busy (measured: 95 % at 8)


def model_time(c: Candidate, n_cells, flops, bytes_min, nq, n_loc, ncomp=1, fields=1, dim=2):
    """Modelled time of one action.

    Thread-per-cell: one thread per cell in 32-cell warp chunks; the machine is
    full at WARPS_TO_FILL_SM warps per SM, and the last round of chunks is the
    tail: eta = warps / (W ceil(warps / W)), W = SMs x WARPS_TO_FILL_SM.
    Cells-per-CTA: ceil(n_cells / C) CTAs of 256 threads over SMs x resident
    slots (resident CTAs per SM from the shared-memory plan, at most 4), the
    same fill/tail factor over slots (a last round at most half full counts as
    1/split of a round plus its gather: the FP64 kernel's tail split), times the
    lane efficiency of its two phases, whose idle lanes co-resident CTAs partly
    fill."""
    t_mem = bytes_min / (HBM_GBS * 1e9)
    if c.kernel == 0:
        warps = max(1, math.ceil(n_cells / 32))
        full = N_SMS * WARPS_TO_FILL_SM
        eta = warps / (full * math.ceil(warps / full))
        rounds = math.ceil(warps / full)
    else:
        smem = _coop_total_bytes(n_loc, nq, dim, ncomp, c.tile_cells, fields, tables_global=c.tables_global)
        resident = max(1, min(4, SMEM_PER_SM // max(smem, 1)))
        ctas = max(1, math.ceil(n_cells / c.tile_cells))
        slots = N_SMS * resident
        eta_par = ctas / (slots * math.ceil(ctas / slots))
        # the FP64 kernel's tail split: with one unit per take (C not a multiple of
        # 32, or 32), the T units of a last round that is at most half full are run
        # as `split` items of 1/split of the points each, plus the unit's gather
        # (about 5 % of a unit), instead of a whole round
        if c.tile_cells % 32 != 0 or c.tile_cells == 32:
            T = ctas % slots
            if T > 0 and 2 * T <= slots:
                split = min(nq, slots // T)
                if split > 1:
                    eta_par = (ctas / slots) / (ctas // slots + 1.0 / split + TAIL_GATHER)
        lanes = 0.5 * eta_simd(c.tile_cells * nq) + 0.5 * eta_simd(c.tile_cells * n_loc)
        eta = eta_par * (1.0 - (1.0 - lanes) / resident)
        rounds = math.ceil(ctas / slots)
    t_fp = flops / (F_PEAK_GFLOPS * 1e9 * max(eta, 1e-3))
    return max(t_fp, t_mem) + T_LAUNCH_S + rounds * T_BATCH_S


def spearman(xs, ys) -> float:
    """Spearman rank correlation (no ties expected)."""
    n = len(xs)
    if n < 2:
        return float("nan")
    rx = {i: r for r, i in enumerate(sorted(range(n), key=lambda i: xs[i]))}
    ry = {i: r for r, i in enumerate(sorted(range(n), key=lambda i: ys[i]))}
    d2 = sum((rx[i] - ry[i]) ** 2 for i in range(n))
    return 1.0 - 6.0 * d2 / (n * (n * n - 1))


_CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")


def _load_cache():
    try:
        with open(_CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache):
    os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
    tmp = _CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE_PATH)


def tune(make_plan, u, key: str, kind, dim, degree, top_b: int = 9, reps: int = 5, use_cache=True,
         time_all: bool = False):
    """Pick the fastest launch configuration for one problem.

    ``make_plan(candidate)`` builds a Plan for the candidate; ``u`` is the input.
    Returns (best Candidate, report dict)."""
    import torch
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache and not time_all:
        c = cache[key]
        return Candidate(c["kernel"], c["tile_cells"]), {"cached": True}
    probe = make_plan(Candidate(1, 1))
    nq, n_loc, ncomp = probe.info.nq, probe.info.n_loc, probe.info.ncomp
    flops, bytes_min, n_cells = probe.flops(), probe.info.bytes_min, probe.mesh.n_cells
    del probe
    cands = candidates(kind, dim, degree, nq, n_loc, ncomp)
    mt = lambda c: model_time(c, n_cells, flops, bytes_min, nq, n_loc, ncomp, dim=dim)  # noqa: E731
    ranked = sorted(cands, key=mt)
    chosen = ranked if time_all else ranked[:top_b]
    measured = {}
    stream = torch.cuda.current_stream()
    for c in chosen:
        plan = make_plan(c)
        y = torch.empty_like(u)
        for _ in range(2):
            plan.apply(u, y)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.apply(u, y)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        measured[c] = statistics.median(ts)
    best = min(measured, key=measured.get)
    report = {"candidates": [c.label() for c in ranked],
              "model_s": {c.label(): mt(c) for c in ranked},
              "measured_s": {c.label(): t for c, t in measured.items()}, "best": best.label()}
    if len(measured) >= 3:
        cs = list(measured)
        report["spearman"] = spearman([mt(c) for c in cs], [measured[c] for c in cs])
    if use_cache:
        cache = _load_cache()
        cache[key] = {"kernel": best.kernel, "tile_cells": best.tile_cells}
        _save_cache(cache)
    return best, report
