"""Domain decomposition on CPU processes: the process grid, the face exchange
and the FP64 global sums of paper_2602_14450_gb300.dd, driving float64
sub-lattices (oracle.subdomain), must reproduce the undivided operator of
Eq. 1 / Eq. 4 and the undivided BiCGStab solve.

In-process ranks (LocalComm) cover many grids cheaply; separate gloo
processes (DistComm, world sizes 2 and 4) cover the real message path.
"""

import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from oracle import solvers as S
from oracle import subdomain as SD
from oracle import wilson as W
from paper_2602_14450_gb300 import dd, synth

BC = (1, 1, 1, -1)
KAPPA = 0.12
DIMS = (4, 4, 8, 8)


def _fields(dims=DIMS):
    return synth.gauge_random(dims, 0.5, seed=13), synth.gaussian_source(dims, seed=14)


# ------------------------------------------------------------------ grid logic

def test_rank_coordinates_round_trip_and_neighbours():
    grid = (2, 1, 2, 4)
    p = dd.Partition((8, 4, 8, 16), grid, 0)
    assert p.size == 16
    seen = set()
    for r in range(p.size):
        c = dd.Partition.coords_of(grid, r)
        assert dd.Partition.rank_of(grid, c) == r
        seen.add(c)
        q = dd.Partition((8, 4, 8, 16), grid, r)
        for mu in range(4):
            up, dn = q.neighbour(mu, +1), q.neighbour(mu, -1)
            cu = dd.Partition.coords_of(grid, up)
            assert cu[mu] == (c[mu] + 1) % grid[mu] and all(cu[n] == c[n] for n in range(4) if n != mu)
            assert dd.Partition((8, 4, 8, 16), grid, up).neighbour(mu, -1) == r
            if grid[mu] == 1:
                assert up == dn == r
    assert len(seen) == 16


def test_blocks_tile_the_lattice_once():
    dims, grid = (4, 4, 8, 8), (2, 2, 1, 2)
    cover = torch.zeros(tuple(reversed(dims)), dtype=torch.int32)
    for r in range(8):
        p = dd.Partition(dims, grid, r)
        cover[p.block()] += 1
        assert p.local_dims == (2, 2, 8, 4)
        assert p.face_sites(3) == 2 * 2 * 8 // 2
    assert torch.all(cover == 1)


def test_partition_rejects_odd_or_uneven_splits():
    with pytest.raises(ValueError):
        dd.Partition((4, 4, 6, 8), (1, 1, 2, 1), 0)      # local z extent 3
    with pytest.raises(ValueError):
        dd.Partition((4, 4, 4, 8), (1, 1, 1, 3), 0)      # 8 does not split into 3
    with pytest.raises(ValueError):
        dd.Partition((4, 4, 4, 8), (1, 1, 1, 2), 2)      # rank outside the grid


def test_choose_grid_splits_t_then_z():
    assert dd.choose_grid((32, 32, 32, 64), 4) == (1, 1, 1, 4)
    assert dd.choose_grid((32, 32, 32, 64), 64) == (1, 1, 2, 32)
    assert dd.choose_grid((8, 8, 8, 4), 4) == (1, 1, 2, 2)
    with pytest.raises(ValueError):
        dd.choose_grid((2, 2, 2, 2), 2)


# ----------------------------------------------------------- in-process ranks

def _domain_set(u, grid, dims=DIMS, bc=BC):
    parts = [dd.Partition(dims, grid, r) for r in range(dd.Partition(dims, grid, 0).size)]
    doms = [SD.SubDomain(p.scatter_gauge(u), KAPPA, grid, p.coords, bc) for p in parts]
    return parts, dd.DomainSet(doms, dd.LocalComm(parts))


GRIDS = [(1, 1, 1, 2), (1, 1, 2, 2), (2, 2, 1, 1), (1, 2, 1, 4), (2, 2, 2, 2), (1, 1, 1, 4)]


@pytest.mark.parametrize("grid", GRIDS)
def test_split_hop_equals_eq1(grid):
    u, psi = _fields()
    parts, ds = _domain_set(u, grid)
    for p in (0, 1):
        xs = [W.restrict(q.scatter_field(psi), 1 - p) for q in parts]
        outs = ds.new_vectors()
        dd.hop(ds, p, xs, outs, a=-0.5, b=2.0, ys=[q.scatter_field(psi) for q in parts])
        got = dd.Partition.gather_field(outs, [q.block() for q in parts])
        want = -0.5 * W.hop_pq(u, psi, p, BC) + 2.0 * W.restrict(psi, p)
        assert torch.allclose(got, want, rtol=0, atol=1e-13 * want.abs().max().item())


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (-1, 1, -1, 1)])
def test_split_eo_operator_equals_eq4_with_boundary_phases(bc):
    u, psi = _fields()
    parts, ds = _domain_set(u, (2, 1, 2, 2), bc=bc)
    xs = [W.restrict(q.scatter_field(psi), 0) for q in parts]
    outs, tmps = ds.new_vectors(), ds.new_vectors()
    dd.eo_operator(ds, xs, outs, tmps)
    got = dd.Partition.gather_field(outs, [q.block() for q in parts])
    want = W.eo_operator(u, W.restrict(psi, 0), KAPPA, bc)
    assert torch.allclose(got, want, rtol=0, atol=1e-13 * want.abs().max().item())


def test_split_dot_is_the_global_fp64_sum():
    u, psi = _fields()
    parts, ds = _domain_set(u, (1, 1, 2, 2))
    a = [q.scatter_field(psi) for q in parts]
    b = [q.scatter_field(2j * psi + 1) for q in parts]
    (z,) = dd.dot(ds, [(a, b)])
    want = S.dot(psi, 2j * psi + 1)
    assert abs(z - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("grid", [(1, 1, 1, 4), (2, 2, 1, 2)])
def test_split_bicgstab_equals_undivided(grid):
    u, psi = _fields()
    parts, ds = _domain_set(u, grid)
    b = W.eo_source(u, psi, KAPPA, BC)
    xs = ds.new_vectors()
    it, res = dd.bicgstab(ds, [q.scatter_field(b) for q in parts], xs, 1e-12)
    x = dd.Partition.gather_field(xs, [q.block() for q in parts])
    x0, info = S.bicgstab(lambda v: W.eo_operator(u, v, KAPPA, BC), b, 1e-12)
    assert res <= 1e-12 and it == info.iterations
    assert S.norm(x - x0) <= 1e-13 * S.norm(x0)
    # the full solution through Eq. 5 solves Eq. 3
    xi = W.eo_reconstruct(u, x, psi, KAPPA, BC)
    assert S.norm(psi - W.dirac(u, xi, KAPPA, BC)) <= 1e-11 * S.norm(psi)


# ------------------------------------------------------------ gloo processes

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, grid, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u, psi = _fields()
        part = dd.Partition(DIMS, grid, rank)
        dom = SD.SubDomain(part.scatter_gauge(u), KAPPA, grid, part.coords, BC)
        ds = dd.DomainSet([dom], dd.DistComm(part))
        errs = {}
        for p in (0, 1):
            x = W.restrict(part.scatter_field(psi), 1 - p)
            (o,) = ds.new_vectors()
            dd.hop(ds, p, [x], [o])
            want = part.scatter_field(W.hop_pq(u, psi, p, BC))
            errs[f"hop{p}"] = (o - want).abs().max().item() / want.abs().max().item()
        b = W.eo_source(u, psi, KAPPA, BC)
        (x,) = ds.new_vectors()
        it, res = dd.bicgstab(ds, [part.scatter_field(b)], [x], 1e-12)
        x0, info = S.bicgstab(lambda v: W.eo_operator(u, v, KAPPA, BC), b, 1e-12)
        xb = part.scatter_field(x0)
        errs["solve"] = (S.norm(x - xb) / S.norm(x0), it, info.iterations, res)
        out[rank] = errs
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,grid", [(2, (1, 1, 1, 2)), (4, (1, 1, 2, 2))])
def test_gloo_ranks_reproduce_undivided_operator_and_solve(world, grid):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, grid, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert sorted(res) == list(range(world))
    for r, e in res.items():
        assert e["hop0"] <= 1e-13 and e["hop1"] <= 1e-13, (r, e)
        rel, it, it0, rr = e["solve"]
        assert it == it0 and rr <= 1e-12, (r, e)
        assert rel <= 1e-13, (r, e)   # this rank's share of the global relative error
