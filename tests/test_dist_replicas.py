"""The multi-GPU path of the bench is replicas only: every rank runs its own
evaluation, the timing is the slowest rank's, the throughput counts every
rank's particles, and only rank 0 prints.  These run as two gloo processes on
the CPU (no GPU, no collective on the data path)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        # each replica timed its own steps; the job is as slow as the slowest
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        rate = bench.job_throughput(1000, 5, ws, t)

        class Args:
            steps, warmup = 1, 0
        out = io.StringIO()
        with redirect_stdout(out):
            rc = bench.run_reference(Args, ws, rank) if rank != 0 else 0
        queue.put((rank, t, rate, rc, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_count_all_particles():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, rc, printed in res:
        assert t == 2.0                      # max over ranks, on every rank
        assert rate == 1000 * 5 * ws / 2.0   # whole-job particles / slowest time
        assert rc == 0
        if rank != 0:
            assert printed == ""             # the reference arm: rank 0 alone works


def test_single_process_has_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(10, 2, 1, 4.0) == 5.0
