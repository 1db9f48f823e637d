"""The multi-GPU path is replicas only: each rank measures its own Monte-Carlo run and the
reported throughput is the total over ranks divided by the slowest rank's time.  The
aggregation runs here as two gloo ranks on the CPU."""
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
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [40.0, 55.0][rank]
    value, frames, ms_max = bench.replica_throughput(local_ms, spots_per_step=1000, steps=10,
                                                      world=world, dev=torch.device("cpu"))
    q.put((rank, value, frames, ms_max))
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, frames, ms_max in out:
        assert ms_max == 55.0
        assert abs(value - 2 * 1000 * 10 / 0.055) < 1e-6 * value
        assert abs(frames - 2 * 10 / 0.055) < 1e-9 * frames


def test_single_rank_needs_no_process_group():
    value, frames, ms_max = bench.replica_throughput(20.0, 500, 4, 1, torch.device("cpu"))
    assert ms_max == 20.0 and abs(value - 500 * 4 / 0.02) < 1e-6
