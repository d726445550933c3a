"""The multi-rank host path of bench.py on CPU ranks (gloo, world size 2):
replicas run independent estimates with distinct request ids and the
whole-job rate is all ranks' estimates over the slowest rank's time."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    rate, max_ms = bench.whole_job_rate(local_ms, 10, world, "cpu")
    q.put((rank, rate, max_ms))
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, max_ms in out:
        assert max_ms == 250.0
        assert rate == pytest.approx(2 * 10 / 0.25)


def test_single_rank_rate_needs_no_process_group():
    import bench
    rate, ms = bench.whole_job_rate(200.0, 20, 1, "cpu")
    assert rate == pytest.approx(100.0) and ms == 200.0
