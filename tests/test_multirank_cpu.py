"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1).

The filters do not shard (replicas only: every rank runs the whole workload
on its own GPU); what crosses ranks is the timing reduction.  Checked here:
the slowest rank's time reaches every rank, the barrier releases both, the
whole-job rate counts every rank's keys over that time, and the reference arm
runs on rank 0 only.
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, local = bench.dist_env()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, w)  # this rank's timed milliseconds
        bench.barrier(w)
        v = bench.whole_job_rate(w, keys_per_step=1_000_000, steps=4, total_ms=t)
        # the reference arm: rank 0 alone runs and prints (a tiny sample here)
        out = io.StringIO()
        printed = None
        if rank != 0:
            with contextlib.redirect_stdout(out):
                bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), bench.WORKLOADS["1MiB"], "1MiB")
            printed = out.getvalue()
        q.put((rank, w, r, local, t, v, printed))
    finally:
        dist.destroy_process_group()


def test_two_ranks_timing_reduction_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, local, t, v, printed in res:
        assert (w, r, local) == (2, rank, rank)
        assert t == 15.0  # the slower rank's time, on both ranks
        assert v == pytest.approx(2 * 1_000_000 * 4 / 15e-3 / 1e9)
    assert res[1][6] == ""  # rank 1 prints nothing in the reference arm
