"""The benchmark's multi-rank host logic on CPU (two `gloo` ranks, no GPU):
every rank advances its own box, the whole-job rate counts the units of all
ranks over the slowest rank's time, and the reference arm runs on rank 0
alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(seconds[rank], dist, "cpu")
    rate = bench.whole_job_rate(1000.0, seconds[rank], world, dist, "cpu")
    queue.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_whole_job_rate_counts_every_rank_over_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    world, seconds = 2, [0.5, 2.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, seconds, queue)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(queue.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in results:
        assert slowest == 2.0
        assert rate == pytest.approx(world * 1000.0 / 2.0)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(500.0, 2.0, 1) == 250.0


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
