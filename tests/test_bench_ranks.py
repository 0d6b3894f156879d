"""The N > 1 path of bench.py as two gloo ranks on the CPU: weak-scaling
replicas get distinct seeded batches of the same shape, every time is
reduced to the slowest rank, and the whole-job rate counts all ranks' units
against that time."""
import os
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    params, t, desc = bench.workload("batch", rank)
    t_local = 1.0 + rank  # rank 1 is the slow one
    t_max = bench.reduce_max(t_local, world, "cpu")
    rate = bench.job_rate(t.size, world, 2, t_max)
    q.put((rank, float(params[0]["q"]), float(t[0, 0]), t.shape, desc["workload"], t_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, q0, t0, s0, w0, m0, v0), (r1, q1, t1, s1, w1, m1, v1) = out
    assert (r0, r1) == (0, 1)
    assert s0 == s1 == (64, 10_000) and w0 == w1          # same workload shape per rank
    assert q0 != q1 and t0 != t1                           # distinct seeds
    assert m0 == m1 == 2.0                                 # the slowest rank's time
    assert v0 == v1 == 64 * 10_000 * 2 * 2 / 2.0            # both ranks' units over that time


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(100, 1, 4, 2.0) == 200.0
    assert np.isclose(bench.job_rate(640_000, 8, 2, 20.0), 512_000.0)
