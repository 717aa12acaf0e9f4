"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective).  The step time is the slowest rank's; the value counts every
rank's work; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [3.0, 5.0][rank]                       # rank 1 is the slow one
        t = bench.reduce_max(ms, world, "cpu")
        v = bench.job_value(2.0e9, world, t)
        # reference arm: rank 1 returns at once without running the oracle
        class A:
            warmup, steps = 3, 1
        ref = bench.run_reference(A(), rank, world) if rank == 1 else None
        q.put((rank, t, v, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v, ref in res:
        assert t == 5.0                                  # max over ranks
        assert abs(v - 2 * 2.0e9 / 5e-3 / 1e9) < 1e-9    # whole-job GFLOP/s
        assert ref is None
