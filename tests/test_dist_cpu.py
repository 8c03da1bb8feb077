"""The multi-rank bench path on CPU (gloo, world size 2): every rank renders its own frame (weak
scaling, no data-path collective); the job's time per step is the slowest rank's, and the whole-job
throughput counts every rank's pixels."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [10.0 + 5.0 * rank, 3.0 - rank]          # rank 1 is slower in the first figure
    got = bench.max_over_ranks(local, world)
    dist.barrier()
    q.put((rank, got, bench.whole_job_mpix_s(world, 1920 * 1080, got[0])))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [15.0, 3.0]                      # max over ranks, figure by figure
        assert value == pytest.approx(2 * 1920 * 1080 / 15e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.whole_job_mpix_s(1, 2_000_000, 2.0) == pytest.approx(1000.0)
