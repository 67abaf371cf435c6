"""Host logic of the multi-rank benchmark path on CPU: two gloo ranks (127.0.0.1) agree on the slowest
rank's timings and the whole-job throughput; the reference arm runs on rank 0 only."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [100.0 + 10 * rank, 5.0 - rank, 7.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, world)
    rate = bench.job_rate(1e9, world, 4, got[0] * 1e-3)
    out.put((rank, got, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [110.0, 5.0, 14.0]
        # 2 ranks x 1e9 units x 4 steps in 0.110 s
        assert abs(rate - 2 * 1e9 * 4 / 0.110 / 1e9) < 1e-9


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps, gpus, ref_seconds, workload = 3, 2, 2, 1.0, "cone512_jitter"

    assert bench.run_reference(A()) == 0
