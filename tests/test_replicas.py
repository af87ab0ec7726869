"""The multi-process path of bench.py without a GPU: N independent replicas (one per rank, no
collective on the data path), the job time is the slowest rank's and the value counts every
rank's sites. Two gloo ranks on the CPU, rendezvous on 127.0.0.1."""
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


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(torch, dist, times[rank], torch.device("cpu"))
        out[rank] = (t, bench.replicas_mlups(world, 1000, 10, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_sites():
    world, times = 2, [0.25, 0.5]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    t, value = res[0]
    assert t == 0.5
    assert value == pytest.approx(2 * 1000 * 10 / 0.5 / 1e6)


def test_replica_value_is_weak_scaling():
    assert bench.replicas_mlups(4, 2 ** 24, 100, 1.0) == pytest.approx(4 * bench.replicas_mlups(1, 2 ** 24, 100, 1.0))
