"""One MapElites repertoire shared by several ranks (one GPU each).

Algorithm 3 keeps a single repertoire; the paper's loop feeds it from one
batch per iteration.  Across ranks the topologies of a step are independent
and the grid factors are read-only, so each rank proposes and evaluates its
own share of the step's candidates.  One exchange per step then keeps the
repertoires identical without a broadcast: an all-gather of every rank's
(genome, fitness, cell) rows, after which every rank inserts the gathered
batch, in rank order, with the same deterministic scatter insert
(tto_archive_insert: per cell the best fitness wins, the lowest gathered index
on ties, strict improvement over the elite).  Since the insert depends only on
the gathered batch and the archive, and every rank holds the same archive
before the step, every rank holds the same archive after it.

Each rank draws its proposals from its own Philox key (``rank_key``), so the
ranks' candidates differ while every draw stays reproducible.

The exchange packs a rank's rows into one int32 tensor [B][width + 2]
(genome, the fitness bits, the cell) so a step needs one collective.  With
the NCCL backend the tensor stays on the device; with gloo (the CPU tests) it
goes through host memory.
"""
from __future__ import annotations

from . import FIT_WORKLOAD, PREC_FP32, DEFAULT_MUTATION

_KEY_MUL = 0x9E3779B97F4A7C15  # odd 64-bit constant: distinct keys for distinct ranks


def rank_key(seed: int, rank: int) -> int:
    """Philox key of a rank's proposals in a shared search: the shared seed
    with the rank mixed in (rank 0 keeps the seed)."""
    return (int(seed) ^ (int(rank) * _KEY_MUL)) & 0xFFFFFFFFFFFFFFFF


def pack_rows(topo, fitness, cell):
    """[B][w] int32 genomes, [B] float32 fitness and [B] int32 cells as one
    int32 tensor [B][w + 2] (the fitness carried as its bit pattern)."""
    import torch
    return torch.cat([topo.to(torch.int32), fitness.to(torch.float32).contiguous().view(torch.int32)[:, None],
                      cell.to(torch.int32)[:, None]], dim=1).contiguous()


def unpack_rows(rows):
    """Inverse of :func:`pack_rows`: (genomes, fitness, cells)."""
    import torch
    w = rows.shape[1] - 2
    return (rows[:, :w].contiguous(), rows[:, w].contiguous().view(torch.float32),
            rows[:, w + 1].contiguous())


def gather_rows(rows, group=None):
    """All-gather the ranks' packed rows (every rank the same row count),
    concatenated in rank order.  One collective; on a gloo group the rows go
    through host memory."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return rows
    world = dist.get_world_size(group)
    if world == 1:
        return rows
    via_host = dist.get_backend(group) == "gloo" and rows.is_cuda
    src = rows.cpu() if via_host else rows
    out = torch.empty((world * src.shape[0], src.shape[1]), dtype=src.dtype, device=src.device)
    dist.all_gather_into_tensor(out, src, group=group)
    return out.to(rows.device) if via_host else out


class SharedArchive:
    """A device archive kept identical across the ranks of ``group``.

    ``step`` runs one shared MapElites iteration: propose ``B`` candidates from
    the local copy with the rank's key, evaluate them exactly, all-gather the
    (genome, fitness, cell) rows of every rank, and insert the gathered batch.
    Returns the gathered rows."""

    def __init__(self, archive, group=None):
        self.archive = archive
        self.grid = archive.grid
        self.group = group

    @property
    def rank(self):
        import torch.distributed as dist
        return dist.get_rank(self.group) if dist.is_available() and dist.is_initialized() else 0

    def step(self, seed, iteration, B, mutation=DEFAULT_MUTATION, precision=PREC_FP32,
             fitness_kind=FIT_WORKLOAD, stream=None):
        a = self.archive
        topo = a.propose(rank_key(seed, self.rank), iteration, B, mutation, stream=stream)
        out = self.grid.evaluate(topo, precision=precision, fitness_kind=fitness_kind, d_split=a.d_split,
                                 d_moved=a.d_moved, d_disc=a.d_disc, stream=stream)
        rows = gather_rows(pack_rows(topo, out["fitness"], out["cell"]), self.group)
        g_topo, g_fit, g_cell = unpack_rows(rows)
        a.insert(g_topo, g_fit, g_cell, stream=stream)
        return rows
