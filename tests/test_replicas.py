"""The multi-GPU path of the benchmark is replicas only: every rank runs the
whole step on its own data and the ranks exchange one number, the maximum
of their step times. Checked here on the CPU with two gloo ranks (no GPU):
the maximum over ranks and the rank / world parsing of bench.py."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, local = bench._dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(10.0 + 5.0 * rank, world)   # rank 1 is the slowest
        out[rank] = m
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist_setup(1) == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_more_gpus_than_ranks_is_refused(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    with pytest.raises(SystemExit):
        bench._dist_setup(2)
