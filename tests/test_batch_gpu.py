"""GPU parity of the batched persistent launch: every problem of a small mixed
batch (forms, dimensions, degrees 1-4, uneven sizes) against the FP64 oracle, with
the automatic kernel choice and with every problem forced onto the cells-per-CTA
code; repeated runs reuse the self-resetting work queue."""

import numpy as np
import pytest
import torch

import oracle
from feinputs import lame_fields, structured_mesh, uniform_field
from feinputs.batch import batch_specs
from feinputs.fields import sinusoid_displacement

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_17471_gb300 as fe
    return fe


def build(fe, specs, kernel=-1, tile=0, tables_global=False):
    problems, refs = [], []
    for s in specs:
        dim, p, N, q = s["dim"], s["degree"], s["N"], s["quad_degree"]
        m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=s["seed"])
        M = fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
        o = oracle.Oracle.from_mesh(m, q)
        pb = {"mesh": M, "quad_degree": q, "kernel": kernel, "tile_cells": tile,
              "tables_global": tables_global}
        if s["form"] == "mass":
            u = uniform_field(m.n_nodes, s["seed"])
            pb.update(kind=fe.MASS)
            ref = o.mass(u)
        elif s["form"] == "elasticity":
            u = uniform_field(m.n_nodes * dim, s["seed"])
            pb.update(kind=fe.ELASTICITY, lam=1.25, mu=1.0)
            ref = o.elasticity(u, 1.25, 1.0)
        else:
            u = sinusoid_displacement(m, s["seed"])
            mu, lam = lame_fields(m.n_cells, s["seed"] + 1)
            pb.update(kind=fe.NH_RESIDUAL, mu_cell=mu, lam_cell=lam)
            ref = o.nh_residual(u, mu, lam)
        pb["u"] = torch.from_numpy(u).cuda()
        problems.append(pb)
        refs.append(ref)
    return problems, refs


@pytest.mark.parametrize("kernel,tile,tables_global", [(-1, 0, False), (1, 8, False), (1, 3, False),
                                                       (1, 5, True)])
def test_batched_matches_oracle(fe, kernel, tile, tables_global):
    specs = batch_specs(count=18, seed=77, cells_min=40, cells_max=2500)
    problems, refs = build(fe, specs, kernel, tile, tables_global)
    batch = fe.Batch(problems)
    assert batch.info["problems"] == len(specs)
    for rep in range(2):
        ys = batch.run()
        torch.cuda.synchronize()
        for s, y, ref in zip(specs, ys, refs):
            err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= TOL, (rep, s, err)
        assert batch.status() == 0


def test_batched_rejects_bad_problems(fe):
    from paper_2506_17471_gb300 import FeError
    specs = batch_specs(count=2, seed=5, cells_min=40, cells_max=100)
    problems, _ = build(fe, specs)
    problems[0]["kernel"] = 0
    problems[0]["mesh"] = problems[0]["mesh"]
    bad = dict(problems[1])
    bad["quad_degree"] = 99
    with pytest.raises(FeError):
        fe.Batch([bad])


def test_full_batch_64_meshes(fe):
    """The benchmark's batch: 64 meshes (2.38M cells, mass / elasticity /
    Neo-Hookean, degrees 1-4, 2D and 3D) in one batched launch; one problem of each
    form and dimension checked in full against the oracle, all for finite output."""
    specs = batch_specs(64)
    problems, meshes = [], []
    for s in specs:
        dim, p, N, q = s["dim"], s["degree"], s["N"], s["quad_degree"]
        m = structured_mesh(dim, N, p, jitter=0.2 if dim == 2 else 0.15, seed=s["seed"])
        M = fe.Mesh(dim, p, m.coords, m.cell2vertex, m.cell2node, m.n_nodes)
        pb = {"mesh": M, "quad_degree": q}
        if s["form"] == "mass":
            u = uniform_field(m.n_nodes, s["seed"])
            pb.update(kind=fe.MASS)
        elif s["form"] == "elasticity":
            u = uniform_field(m.n_nodes * dim, s["seed"])
            pb.update(kind=fe.ELASTICITY, lam=1.25, mu=1.0)
        else:
            u = sinusoid_displacement(m, s["seed"])
            mu, lam = lame_fields(m.n_cells, s["seed"] + 1)
            pb.update(kind=fe.NH_RESIDUAL, mu_cell=mu, lam_cell=lam)
        pb["u"] = torch.from_numpy(u).cuda()
        problems.append(pb)
        meshes.append((m, u, pb))
    batch = fe.Batch(problems)
    assert sum(s["n_cells"] for s in specs) > 2_000_000
    ys = batch.run()
    torch.cuda.synchronize()
    assert batch.status() == 0
    assert all(bool(torch.isfinite(y).all()) for y in ys)
    checked = set()
    for s, y, (m, u, pb) in zip(specs, ys, meshes):
        key = (s["form"], s["dim"])
        if key in checked or s["n_cells"] > 60_000:
            continue
        checked.add(key)
        o = oracle.Oracle.from_mesh(m, s["quad_degree"])
        if s["form"] == "mass":
            ref = o.mass(u, threads=16)
        elif s["form"] == "elasticity":
            ref = o.elasticity(u, 1.25, 1.0, threads=16)
        else:
            ref = o.nh_residual(u, pb["mu_cell"], pb["lam_cell"], threads=16)
        err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= (TOL if s["form"] != "neo_hookean" else 1e-11), (s, err)
    assert len(checked) >= 4
