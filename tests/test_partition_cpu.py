"""Multi-process sharding logic on CPU ranks (gloo, world size 2): cell ranges,
interface sum by all-reduce, and problem sharding.  The per-rank compute is the
oracle on the rank's cell range, so the test needs no GPU."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


@pytest.fixture(scope="module")
def part():
    import __graft_entry__
    __graft_entry__.build_library()   # the package loads the built library on import
    from paper_2506_17471_gb300 import partition
    return partition


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2506_17471_gb300.partition import cell_range
    from feinputs import structured_mesh, uniform_field
    from paper_2506_17471_gb300.partition import interface_sum
    m = structured_mesh(3, 4, 2, jitter=0.15, seed=5)
    o = oracle.Oracle.from_mesh(m, 2)
    u = uniform_field(m.n_nodes * 3, 6)
    c0, c1 = cell_range(m.n_cells, rank, world)
    part = torch.from_numpy(o.elasticity(u, 1.25, 1.0, cells=(c0, c1)))
    interface_sum(part)
    np.save(os.path.join(result_dir, f"y{rank}.npy"), part.numpy())
    dist.destroy_process_group()


def test_cell_ranges_cover_once(part):
    cell_range = part.cell_range
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            ranges = [cell_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        cell_range(10, 2, 2)


def test_problem_sharding_partitions(part):
    problems_of_rank = part.problems_of_rank
    assigned = sorted(p for r in range(3) for p in problems_of_rank(64, r, 3))
    assert assigned == list(range(64))


def test_two_rank_interface_sum_matches_single_domain(part, tmp_path):
    import oracle
    from feinputs import structured_mesh, uniform_field
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    m = structured_mesh(3, 4, 2, jitter=0.15, seed=5)
    o = oracle.Oracle.from_mesh(m, 2)
    ref = o.elasticity(uniform_field(m.n_nodes * 3, 6), 1.25, 1.0)
    for r in range(world):
        y = np.load(tmp_path / f"y{r}.npy")
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
