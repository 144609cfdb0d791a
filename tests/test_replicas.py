"""The multi-GPU path is replicas only (one graph does not shard): N ranks
each run their own graph and bench.py reports the units of all ranks over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 1.5 if rank == 0 else 2.5  # the second replica is slower
    slowest = bench.max_over_ranks(mine, world)
    out[rank] = (slowest, bench.replica_throughput(1000, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_all_units_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2.5, 2000 / 2.5)


def test_one_process_is_unchanged():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_throughput(64154 * 8, 1, 0.04) == pytest.approx(64154 * 8 / 0.04)
