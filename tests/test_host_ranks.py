"""The multi-rank timing of bench.py on CPU: two gloo ranks with different
timed regions report the slowest rank's time and the units all ranks
processed over it (weak scaling, one replica per rank)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 300.0, 80.0][rank]
        t, rate = bench.whole_job_rate(elapsed, 64 * 3, dist, "cpu")
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_whole_job_rate_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([120.0, 300.0, 80.0][:world])
    for rank, t, rate in out:
        assert t == slowest
        assert rate == pytest.approx(64 * 3 * world / (slowest * 1e-3))


def test_whole_job_rate_single_process():
    t, rate = bench.whole_job_rate(250.0, 64)
    assert t == 250.0 and rate == pytest.approx(64 / 0.25)
