"""Host logic of the autotuner (no GPU): candidate space, pruning, cost model,
Spearman rank correlation (the paper's Eq. "spearmann_rho")."""

import math

import pytest


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2506_17471_gb300 import autotune
    return autotune


def test_eta_simd_closed_form(at):
    # the paper's eta_simd = N_c N_WI / (32 ceil(N_c N_WI / 32)) with 32-wide groups
    for items in (1, 31, 32, 33, 64, 100):
        assert at.eta_simd(items, 32) == pytest.approx(items / (32 * math.ceil(items / 32)))
    assert at.eta_simd(256) == 1.0 and at.eta_simd(257) == pytest.approx(257 / 512)


def test_candidates_follow_tile_constraint_and_pruning(at):
    from paper_2506_17471_gb300 import _native as N
    cands = at.candidates(N.FE_FORM_ELASTICITY, 3, 4, nq=64, n_loc=35, ncomp=3)
    assert all(c.kernel == 1 for c in cands)          # no thread-per-cell kernel for P4 tets
    assert {c.tables_global for c in cands} == {False, True}
    cands = [c for c in cands if not c.tables_global]
    tiles = [c.tile_cells for c in cands]
    assert tiles == sorted(tiles, reverse=True)
    cmax = max(tiles)
    assert all(any(t == math.ceil(cmax / k) for k in range(1, 64)) for t in tiles)
    for t in tiles:
        assert t == cmax or at.eta_simd(t * 64) >= 0.3
        assert at._coop_total_bytes(35, 64, 3, 3, t, 1, tables_global=False) <= at.SMEM_BUDGET
    assert at._coop_total_bytes(35, 64, 3, 3, cmax + 1, 1, tables_global=False) > at.SMEM_BUDGET
    big = at.candidates(N.FE_FORM_NH_RESIDUAL, 3, 4, nq=125, n_loc=35, ncomp=3)
    assert big and all(c.tables_global for c in big)     # a 140 KB table never goes to shared
    c2 = at.candidates(N.FE_FORM_MASS, 2, 2, nq=9, n_loc=6, ncomp=1)
    assert c2[0].kernel == 0                           # thread-per-cell exists for P2 mass


def test_cost_model_monotone(at):
    c = at.Candidate(0)
    t1 = at.model_time(c, 1000, 1e8, 1e6, 8, 10)
    t2 = at.model_time(c, 1000, 2e8, 1e6, 8, 10)
    assert t2 > t1
    # memory-bound regime: time follows bytes
    t3 = at.model_time(c, 1000, 1.0, 1e9, 8, 10)
    assert t3 == pytest.approx(1e9 / (at.HBM_GBS * 1e9) + at.T_LAUNCH_S + at.T_BATCH_S)
    # a mesh too small to fill the machine favours the cells-per-CTA kernel
    small_tpc = at.model_time(at.Candidate(0), 2000, 1e8, 1e6, 27, 20, 1, dim=3)
    small_coop = at.model_time(at.Candidate(1, 4), 2000, 1e8, 1e6, 27, 20, 1, dim=3)
    assert small_coop < small_tpc


def test_cost_model_tail_split(at):
    """The FP64 cells-per-CTA kernel splits a last round that is at most half full
    by quadrature points, so a few extra units cost a fraction of a round; a last
    round more than half full still costs a whole round."""
    C, n, nq = 10, 20, 27
    resident = max(1, min(4, at.SMEM_PER_SM // at._coop_total_bytes(n, nq, 3, 1, C, 1)))
    slots = at.N_SMS * resident
    c = at.Candidate(1, C)

    def t(units):   # FP64 work in proportion to the units; launch and batch overheads left out
        rounds = -(-units // slots)
        return at.model_time(c, units * C, 1e6 * units, 0.0, nq, n, 1, dim=3) - at.T_LAUNCH_S \
            - rounds * at.T_BATCH_S

    one = t(slots)
    assert t(slots + 3) < 1.2 * one                            # 3 units split min(27, slots/3) ways
    assert t(slots + (3 * slots) // 4) == pytest.approx(2 * one, rel=1e-9)   # no split: a whole round
    assert t(2 * slots) == pytest.approx(2 * one, rel=1e-9)


def test_spearman(at):
    assert at.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == 1.0
    assert at.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == -1.0
    assert at.spearman([1, 2, 3, 4, 5], [2, 1, 4, 3, 5]) == pytest.approx(0.8)
