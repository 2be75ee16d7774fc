"""The shared-repertoire step across ranks (paper_2605_10128_b300.shared_archive)
on CPU: two gloo ranks propose from their own copy of one archive with their
own Philox keys, evaluate with the oracle, exchange (genome, fitness, cell)
rows with the library's all-gather helper and insert the gathered batch with
the oracle's sequential insert (Algorithm 3).  Both ranks must end with the
same archive, equal to one process inserting both ranks' batches in rank
order."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SEED, B, ITERS = 31, 24, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    from oracle import dcflow, mapelites as me
    from synth import config_grid, limits_from_flows
    sg = config_grid("tto30")
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 5))
    return sg, me.ActionTable(sg), me.Archive(8, 8)


def _rows(sg, tab, arch, key, it):
    """One rank's candidates of an iteration as packed int32 rows."""
    from oracle import dcflow, mapelites as me
    from paper_2605_10128_b300.shared_archive import pack_rows
    topo = me.propose(arch, tab, key, it, B, sg.k_max)
    res = [dcflow.evaluate(sg, t) for t in topo]
    fit = torch.tensor([r["fitness"] for r in res], dtype=torch.float32)  # exchanged as FP32
    cell = torch.tensor([r["cell"] for r in res], dtype=torch.int32)
    return pack_rows(torch.from_numpy(topo), fit, cell)


def _insert(arch, rows):
    from paper_2605_10128_b300.shared_archive import unpack_rows
    t, f, c = unpack_rows(rows)
    arch.insert(c.numpy(), f.numpy().astype(np.float64), t.numpy())


def _snapshot(arch):
    return sorted((c, f, tuple(int(x) for x in g)) for c, (f, g) in arch.elites.items())


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2605_10128_b300.shared_archive import gather_rows, rank_key
    sg, tab, arch = _setup()
    sizes = []
    for it in range(ITERS):
        rows = gather_rows(_rows(sg, tab, arch, rank_key(SEED, rank), it))
        sizes.append(int(rows.shape[0]))
        _insert(arch, rows)
    q.put((rank, _snapshot(arch), sizes))
    dist.barrier()
    dist.destroy_process_group()


def test_pack_rows_roundtrip():
    from paper_2605_10128_b300.shared_archive import pack_rows, unpack_rows, rank_key
    t = torch.tensor([[3, -1], [7, 9]], dtype=torch.int32)
    f = torch.tensor([-1.25, -float("inf")], dtype=torch.float32)
    c = torch.tensor([5, 0], dtype=torch.int32)
    t2, f2, c2 = unpack_rows(pack_rows(t, f, c))
    assert torch.equal(t2, t) and torch.equal(c2, c)
    assert f2[0].item() == -1.25 and f2[1].item() == -float("inf")
    assert rank_key(31, 0) == 31 and len({rank_key(31, r) for r in range(8)}) == 8


def test_two_gloo_ranks_keep_one_archive():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, snap0, sizes0), (_, snap1, _) = res
    assert sizes0 == [world * B] * ITERS
    assert snap0 == snap1 and len(snap0) > 1
    # one process inserting both ranks' batches in rank order
    from paper_2605_10128_b300.shared_archive import rank_key
    sg, tab, arch = _setup()
    for it in range(ITERS):
        rows = torch.cat([_rows(sg, tab, arch, rank_key(SEED, r), it) for r in range(world)])
        _insert(arch, rows)
    assert _snapshot(arch) == snap0
