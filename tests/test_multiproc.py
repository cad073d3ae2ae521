"""Host logic of the N>1 benchmark path on CPU: every rank renders its own
replica (no data-path collective); the job's throughput is all ranks'
samples over the slowest rank's time, reduced with a MAX all-reduce.  Run as
two gloo ranks; the reference arm prints only on rank 0."""
import io
import os
import sys
import contextlib

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = [2.0, 5.0][rank]
    value, worst = bench.aggregate(step_ms, 1e9, world, bench.make_reduce_max(world, "cpu"))
    q.put((rank, value, worst))
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, worst in out:
        assert worst == 5.0
        assert value == pytest.approx(2 * 1e9 / 5e-3 / 1e9)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert rc == 0 and buf.getvalue() == ""
