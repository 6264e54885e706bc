"""The N > 1 path of bench.py on the CPU: two ranks over gloo (replicas of the frame, no
data-path collective).  The job's time per step is the slowest rank's, its rate the units of
all ranks over that time; the reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, ms, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + bench.job_rate(ms, 1000, world, "cpu"))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r, ms in ((0, 2.0), (1, 5.0))]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    for rank, ms, value in got:
        assert ms == 5.0                              # the max over ranks, on every rank
        assert value == pytest.approx(2 * 1000 / 5e-3)  # both ranks' units over that time


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(4.0, 1000, 1) == (4.0, 1000 / 4e-3)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
