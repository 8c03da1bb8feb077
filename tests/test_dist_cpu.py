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


def _grad_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2606_23031_gb300 as dv
    # per-octree gradients of this rank's cameras (seeded by rank), shapes of a background and two actors
    g = torch.Generator().manual_seed(100 + rank)
    shapes = [(50, 8), (7, 8), (0, 8), (50, 16, 3), (7, 16, 3), (0, 16, 3)]
    ts = [torch.randn(s, generator=g, dtype=torch.float32) for s in shapes]
    mine = [t.clone() for t in ts]
    dv.allreduce_gradients(ts)
    q.put((rank, [t.numpy() for t in mine], [t.numpy() for t in ts], dv.camera_shard(list(range(6)), rank, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_camera_split_gradient_exchange_gloo():
    """Cameras split across two ranks: each rank's gradients become the sum over both ranks, tensor by
    tensor (empty tensors of a barely seen actor included), and the shards cover every camera once."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, own0, sum0, sh0), (_, own1, sum1, sh1) = res
    for a, b, s0, s1 in zip(own0, own1, sum0, sum1):
        np.testing.assert_array_equal(s0, s1)
        np.testing.assert_allclose(s0, a + b, rtol=1e-6, atol=1e-7)
    assert sorted(sh0 + sh1) == list(range(6)) and not set(sh0) & set(sh1)
