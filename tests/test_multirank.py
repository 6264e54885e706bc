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


def _split_rank(rank, world, port, q):
    """One rank of the points-across-GPUs split on the CPU: the shard's keys from the oracle
    (its global indices), combined by the package's collective step; owner-masked resolve of
    the combined keys, planes added across ranks."""
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import nrv_inputs as I
    import oracle
    from paper_2407_19097_gb300 import split
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = I.trajectory_scene(1500, 35, seed=2)
        view = I.fitted_view(sc, 160, 96)
        lo, hi = split.shard_range(sc.n, rank, world)
        shard = sc.subset(np.arange(lo, hi))
        k = oracle.visibility(shard.xyz, view)
        hit = k != np.uint64(0xFFFFFFFFFFFFFFFF)
        k[hit] += np.uint64(lo)                       # global indices in the low word
        keys = torch.from_numpy(k.view(np.int64).copy())

        def flip(t):
            t.bitwise_xor_(torch.tensor(-(1 << 63), dtype=torch.int64))

        split.combine_keys_(keys, flip=flip)
        comb = keys.numpy().view(np.uint64)
        full = oracle.visibility(sc.xyz, view)
        ok_keys = bool(np.array_equal(comb, full))
        # owner-masked resolve: winners outside [lo, hi) are empty on this rank
        idx = comb & np.uint64(0xFFFFFFFF)
        own = (comb != np.uint64(0xFFFFFFFFFFFFFFFF)) & (idx >= lo) & (idx < hi)
        local = np.where(own, comb - np.uint64(lo), np.uint64(0xFFFFFFFFFFFFFFFF))
        d, m, g = oracle.resolve(local, shard.attr, sc.n_words)
        planes = [torch.from_numpy(d.view(np.int32).astype(np.int64)),
                  torch.from_numpy(m.astype(np.int64)),
                  torch.from_numpy(g.view(np.int32).astype(np.int64))]
        split.combine_planes_(planes)
        fd, fm, fg = oracle.resolve(full, sc.attr, sc.n_words)
        ok_planes = (np.array_equal(planes[0].numpy().astype(np.int32).view(np.uint32), fd) and
                     np.array_equal(planes[1].numpy().astype(np.uint8), fm) and
                     np.array_equal(planes[2].numpy().astype(np.int32).view(np.uint32), fg))
        q.put((rank, ok_keys, ok_planes, int(own.sum()), int(hit.sum())))
    finally:
        dist.destroy_process_group()


def test_points_split_combines_to_the_whole_scene():
    """World size 2 over gloo: shard the points, MIN all-reduce of the sign-flipped keys,
    owner resolve, SUM all-reduce of the planes -- bit-exact against the unsharded oracle."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    for rank, ok_keys, ok_planes, owned, hit in got:
        assert ok_keys, f"rank {rank}: combined keys differ from the whole scene's"
        assert ok_planes, f"rank {rank}: summed planes differ from the whole scene's"
        assert owned > 0 and hit > 0
