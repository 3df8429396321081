"""bench.py's multi-process path on CPU: two gloo ranks, the barrier and the
max-over-ranks timing that the replica runs use (one process per GPU on a
GPU host; the solve itself has no exchange step)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import bench
    r, ws, _ = bench.dist_setup()
    assert (r, ws) == (rank, 2)
    bench.barrier(ws)
    out[rank] = bench.max_over_ranks(1.5 + rank, ws)
    bench.barrier(ws)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_over_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(port, out), nprocs=2, start_method="spawn", join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def _reference_rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import bench
    r, ws, _ = bench.dist_setup()
    # ranks other than 0 leave the reference arm without work
    if r != 0:
        out[rank] = bench.reference_arm(None, r, ws)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_reference_arm_idles_on_other_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_reference_rank, args=(port, out), nprocs=2, start_method="spawn", join=True)
        assert dict(out) == {1: None}
