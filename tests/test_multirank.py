"""The bench's multi-rank path on CPU: two gloo ranks (127.0.0.1), the job
time is the slowest rank's, the value counts every rank's samples, and the
oracle reference arm prints from rank 0 only."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    t = bench.reduce_max_ms(ms, dist, "cpu")
    v = bench.job_msamples_per_s(world, 1_000_000, 10, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == pytest.approx(150.0)
        # 2 ranks x 1e6 samples x 10 steps in 0.15 s
        assert v == pytest.approx(2 * 1e6 * 10 / 0.15 / 1e6)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(12.5, None, "cpu") == 12.5
    assert bench.job_msamples_per_s(1, 4096, 100, 1000.0) == pytest.approx(0.4096)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
