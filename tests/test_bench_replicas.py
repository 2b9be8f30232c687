"""The multi-GPU form of bench.py is independent replicas (the path has no
exchange step on one scene per GPU): CPU checks of its host logic with a
world-size-2 gloo process group -- max-over-ranks timing, the whole-job
throughput, and the reference arm's rank-0-only behaviour."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow replica
        q.put((rank, bench.max_over_ranks(ms, world, device="cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(world))
    assert got == {0: 15.0, 1: 15.0}


def test_replica_throughput_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas x 1000 particles x 10 substeps in 5 ms (max over ranks) -> 4e6 particle-substeps/s
    assert bench.replica_throughput(1000, 10, 2, 5.0) == pytest.approx(4.0e6)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
