"""The bench's several-GPU path runs independent replicas (the workload
does not shard: each scenario is one forest on one GPU); its host logic --
the whole-job rate as all ranks' units over the slowest rank's time, and
the barrier around the timed region -- is checked here with two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.barrier()
    value, t = bench.replica_throughput(1000.0, 2.0 + rank, world)
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_uses_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for rank in range(world):
        value, t = out[rank]
        assert t == 3.0                      # the slower rank's time
        assert value == pytest.approx(1000.0 * 2 / 3.0)


def test_single_process_rate():
    value, t = bench.replica_throughput(500.0, 4.0, 1)
    assert (value, t) == (125.0, 4.0)
