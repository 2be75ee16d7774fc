"""The multi-GPU form of the benchmark on CPU ranks: two gloo processes run
the cross-rank part of bench.py (independent seeds, max-over-ranks timing,
whole-job throughput) exactly as the GPU ranks do, without a device."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]  # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, world, "cpu")
    v = bench.job_throughput(8192, world, 10, m)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    q.put((rank, m, v, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_gpu_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, seeds in res:
        assert m == 180.0  # every rank sees the slowest rank's time
        assert v == pytest.approx(8192 * 2 * 10 / 0.18)  # all ranks' work over that time
        assert len(set(seeds)) == world  # independent searches
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.job_throughput(100, 1, 4, 2000.0) == 200.0
