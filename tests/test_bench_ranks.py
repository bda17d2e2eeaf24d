"""The benchmark's multi-replica host logic on CPU: two gloo ranks, the job's
time is the slowest rank's and the job's rate counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out[rank] = (bench.max_over_ranks(10.0 + 5.0 * rank), bench._dist())
    finally:
        dist.destroy_process_group()


def test_slowest_rank_times_the_job():
    import bench
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        got = dict(out)
    assert got[0][0] == got[1][0] == 15.0          # max over ranks, seen by every rank
    assert got[0][1] == (2, 0) and got[1][1] == (2, 1)  # WORLD_SIZE and RANK as torchrun sets them
    # 2 replicas of 1000 units each in 250 ms (the slowest rank): 8000 units/s for the job
    assert bench.job_rate(1000, 2, 250.0) == pytest.approx(8000.0)
    # without a process group the value is its own maximum
    assert bench.max_over_ranks(3.5) == 3.5
