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


def _reference_line(monkeypatch, capsys, rank, world):
    monkeypatch.setenv("RANK", str(rank))
    monkeypatch.setenv("WORLD_SIZE", str(world))
    monkeypatch.setenv("LOCAL_RANK", str(rank))
    # The oracle's timing itself (a minute of FP64 work here) is stubbed: this
    # checks the arm's host logic and its line, not the oracle.
    monkeypatch.setattr(bench, "oracle_iteration_seconds", lambda X, B, Q, rows: (20.0, 1.0, rows))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1",
                                     "--warmup", "0"])
    rc = bench.main()
    return rc, capsys.readouterr().out


def test_reference_arm_prints_on_rank_0_only(monkeypatch, capsys):
    # Under torchrun the reference arm runs on rank 0 alone; the other ranks
    # exit 0 without work or output.
    rc, out = _reference_line(monkeypatch, capsys, 1, 2)
    assert rc == 0 and out.strip() == ""
    rc, out = _reference_line(monkeypatch, capsys, 0, 2)
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert rc == 0 and len(lines) == 1
    import json
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    # The same workload configuration object as the GPU arm's line.
    assert line["config"] == bench.headline_config("fp16", 2)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] == bench.WORKLOAD.t / (20.0 * (bench.LANCZOS_ITERS + bench.J_WORKLOAD))
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["value"] == line["value"]
