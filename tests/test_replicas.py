"""The multi-GPU path's host logic (independent replicas) on CPU: two gloo
ranks exchange the max of their timings; seeds are disjoint per rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_22984_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 + rank  # the slower rank decides the job's time
        out[rank] = replicas.max_over_ranks(t, dist)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 2.5


def test_max_over_ranks_single_process():
    assert replicas.max_over_ranks(3.0) == 3.0


def test_replica_seeds_are_disjoint():
    seeds = {replicas.replica_seed(r, i) for r in range(8) for i in range(100)}
    assert len(seeds) == 800
    assert replicas.replica_seed(1, 0) >> 32 == 1
    with pytest.raises(ValueError):
        replicas.replica_seed(-1, 0)


def test_whole_job_throughput_counts_every_rank():
    assert replicas.whole_job_throughput(16384, 4, 10, 2.0) == 16384 * 4 * 10 / 2.0
    with pytest.raises(ValueError):
        replicas.whole_job_throughput(1, 1, 1, 0.0)
