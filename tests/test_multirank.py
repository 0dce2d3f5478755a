"""Multi-rank host logic of the benchmark on CPU: world size 2 over gloo.

Each rank transforms its own data (weak scaling); the job's time is the
slowest rank's, taken with an all-reduce MAX after a barrier, and the
whole-job rate counts the units of every rank.  The reference arm runs on
rank 0 only."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(0.5 + rank, world, torch.device("cpu"))
        rate = bench.whole_job_gelems(world, 10, 2e9, t)
        ref_rc = bench.run_reference(None, rank) if rank != 0 else None  # non-zero ranks: no work
        dist.barrier()
        q.put((rank, t, rate, ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate, ref_rc in res:
        assert t == 1.5                      # max over ranks of 0.5 + rank
        assert abs(rate - 2 * 10 * 2e9 / 1.5 / 1e9) < 1e-9
    assert res[1][3] == 0                    # rank 1 of the reference arm returns at once


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25
    assert bench.whole_job_gelems(1, 4, 1e9, 2.0) == 2.0
