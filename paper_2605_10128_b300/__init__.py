"""B300-native DC N-1 topology evaluation and MapElites search.

Thin Python layer over the C ABI of ``libtto.so`` (``include/tto.h``).  Torch is
used only for device memory and streams; all computation runs in the library's
CUDA kernels.  There is no CPU fallback: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    TTOError, PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_TF32X3, PREC_FP16X3, FIT_WORKLOAD, FIT_F1, FIT_F2,
    SCREEN_SCORE, SCREEN_CELL_GAIN,
)

DEFAULT_MUTATION = (0.2, 0.2, 0.5, 0.1, 2.0)  # p_add, p_remove, p_change, p_identity, N_mutmean


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise TTOError(_lib.TTO_E_CUDA, "no CUDA device")
    return torch


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class Grid:
    """A grid resident on the device, created from a grid description (any
    object with the fields of ``synth.SynthGrid``)."""

    def __init__(self, desc, device: int = 0):
        _torch()
        self.device = device
        self._h = _lib.tto_grid_create(desc, device)
        info = _lib.tto_grid_info(self._h)
        self.n_branch = info["n_branch"]
        self.n_monitored = info["n_monitored"]
        self.n_outage = info["n_outage"]
        self.n_time = info["n_time"]
        self.k_max = info["k_max"]
        self.n_action = info["n_action"]
        self.n_disc, self.n_dslot = _lib.tto_grid_disc_info(self._h)
        self.genome_width = self.k_max + self.n_dslot

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            _lib.tto_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def base_flows(self) -> np.ndarray:
        return _lib.tto_grid_base_flows(self._h, self.n_time, self.n_branch)

    def set_limits(self, limit):
        _lib.tto_grid_set_limits(self._h, limit)

    def reserve(self, max_batch: int, n_t: int | None = None):
        _lib.tto_grid_reserve(self._h, max_batch, self.n_time if n_t is None else n_t)

    def evaluate(self, topo, timesteps=None, precision=PREC_FP32, fitness_kind=FIT_WORKLOAD,
                 d_split=8, d_moved=8, metrics=False, fmax=False, stream=None, out=None, d_disc=1):
        """Exact N-1 evaluation of ``topo`` (CUDA int32 tensor [B][k_max +
        n_dslot]: split actions, then disconnections).  Returns a dict of CUDA
        tensors: fitness, desc, cell, island and, when asked, metrics [B][4]
        and fmax [B][n_t][n_monitored]."""
        torch = _torch()
        B = int(topo.shape[0])
        if topo.dtype != torch.int32 or not topo.is_cuda or topo.shape[1] != self.genome_width:
            raise TTOError(_lib.TTO_E_ARG, "topo must be a CUDA int32 tensor [B][k_max + n_dslot]")
        topo = topo.contiguous()
        n_t = self.n_time if timesteps is None else len(timesteps)
        dev = topo.device
        if out is None:
            out = dict(fitness=torch.empty(B, dtype=torch.float32, device=dev),
                       desc=torch.empty(B, 2, dtype=torch.int32, device=dev),
                       cell=torch.empty(B, dtype=torch.int32, device=dev),
                       island=torch.empty(B, dtype=torch.uint8, device=dev))
            if metrics:
                out["metrics"] = torch.empty(B, 4, dtype=torch.float32, device=dev)
            if fmax:
                out["fmax"] = torch.empty(B, n_t, self.n_monitored, dtype=torch.float32, device=dev)
        o = _lib.EvalOpts(precision, fitness_kind, d_split, d_moved, d_disc)
        _lib.tto_evaluate_batch(self._h, topo, B, timesteps, o, out["fitness"], out.get("desc"),
                                out.get("cell"), out.get("island"), out.get("metrics"),
                                out.get("fmax"), _stream(stream))
        out["_topo"] = topo
        return out

    def worst_k(self, topo, k=20, timesteps=None, all_energy=False, stream=None):
        """Worst-k N-1 export: per topology the k outages (indices into the
        outage list, -1 = none) of largest overload energy and those energies;
        with all_energy, also every outage's energy [n][n_outage] (NaN where the
        outage islands the topology or its branch is open)."""
        torch = _torch()
        n = int(topo.shape[0])
        if topo.dtype != torch.int32 or not topo.is_cuda or topo.shape[1] != self.genome_width:
            raise TTOError(_lib.TTO_E_ARG, "topo must be a CUDA int32 tensor [n][k_max + n_dslot]")
        topo = topo.contiguous()
        dev = topo.device
        idx = torch.empty(n, k, dtype=torch.int32, device=dev)
        val = torch.empty(n, k, dtype=torch.float32, device=dev)
        allE = torch.empty(n, self.n_outage, dtype=torch.float32, device=dev) if all_energy else None
        _lib.tto_worst_k(self._h, topo, n, timesteps, k, idx, val, allE, _stream(stream))
        out = {"outage": idx, "energy": val}
        if allE is not None:
            out["all_energy"] = allE
        return out

    def busbar(self, topo, timesteps=None, bmax=False, stream=None):
        """Busbar outages of each topology: lambda_b [B] (NaN where the
        topology islands), the islanding busbar outages [B] and, when asked,
        bmax [B][n_t][n_monitored]."""
        torch = _torch()
        B = int(topo.shape[0])
        if topo.dtype != torch.int32 or not topo.is_cuda or topo.shape[1] != self.genome_width:
            raise TTOError(_lib.TTO_E_ARG, "topo must be a CUDA int32 tensor [B][k_max + n_dslot]")
        topo = topo.contiguous()
        dev = topo.device
        n_t = self.n_time if timesteps is None else len(timesteps)
        out = {"lambda_b": torch.empty(B, dtype=torch.float32, device=dev),
               "n_island": torch.empty(B, dtype=torch.int32, device=dev)}
        if bmax:
            out["bmax"] = torch.empty(B, n_t, self.n_monitored, dtype=torch.float32, device=dev)
        _lib.tto_evaluate_busbar(self._h, topo, B, timesteps, out["lambda_b"], out["n_island"], out.get("bmax"),
                                 _stream(stream))
        return out

    def busbar_reference(self, timesteps=None, stream=None):
        """Compute lambda_b of the unsplit topology for lambda_f2 evaluations."""
        _lib.tto_grid_busbar_reference(self._h, timesteps, _stream(stream))

    def sync_status(self, stream=None):
        _lib.tto_grid_sync_status(self._h, _stream(stream))

    def debug_bounded_wait(self, cycles=2_000_000, stream=None):
        """Make one bounded device wait run out (timeout-path test)."""
        _lib.tto_debug_bounded_wait(self._h, cycles, _stream(stream))

    def autotune(self, B, n_t=None, precision=PREC_FP32, stream=None):
        """Time the sweep tile variants on this grid and keep the fastest;
        returns (variant, [ms per variant])."""
        return _lib.tto_grid_autotune(self._h, B, self.n_time if n_t is None else n_t, precision,
                                      _stream(stream))

    def set_sweep_shape(self, precision, shape):
        _lib.tto_grid_set_sweep_shape(self._h, precision, shape)

    def profile(self, enable=True):
        """Start (clearing the record) or stop per-stage event timing."""
        _lib.tto_grid_profile(self._h, enable)

    def profile_read(self):
        """([split update ms, N-1 sweep ms, reduction ms, busbar sweep ms]
        summed, number of calls)."""
        return _lib.tto_grid_profile_read(self._h)


class Archive:
    """Device-resident MapElites archive (one elite per cell)."""

    def __init__(self, grid: Grid, d_split: int, d_moved: int, d_disc: int = 1):
        self.grid = grid
        self.d_split = d_split
        self.d_moved = d_moved
        self.d_disc = d_disc
        self.cells = d_split * d_moved * d_disc
        self._h = _lib.tto_archive_create(grid.handle, d_split, d_moved, d_disc)

    def close(self):
        if self._h is not None:
            _lib.tto_archive_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self):
        return _lib.tto_archive_export(self._h, self.cells, self.grid.genome_width)

    def load(self, fitness, genome, filled):
        _lib.tto_archive_import(self._h, fitness, genome, filled)

    def epoch_export(self, k=20, stream=None):
        """Queue the end-of-epoch hand-over: a snapshot of the archive and the
        worst-k N-1 cases of every cell, copied to pinned host tensors while
        later work on the stream runs.  Returns the host tensors (fitness,
        genome, filled, worst_outage, worst_energy), complete after
        epoch_wait()."""
        torch = _torch()
        gw = self.grid.genome_width
        out = {"fitness": torch.empty(self.cells, dtype=torch.float32).pin_memory(),
               "genome": torch.empty(self.cells, gw, dtype=torch.int32).pin_memory(),
               "filled": torch.empty(self.cells, dtype=torch.uint8).pin_memory(),
               "worst_outage": torch.empty(self.cells, max(k, 1), dtype=torch.int32).pin_memory(),
               "worst_energy": torch.empty(self.cells, max(k, 1), dtype=torch.float32).pin_memory()}
        _lib.tto_epoch_export(self._h, k, out["fitness"], out["genome"], out["filled"], out["worst_outage"],
                              out["worst_energy"], _stream(stream))
        self._pending_export = out  # keep the buffers alive until the copy completes
        return out

    def epoch_wait(self):
        _lib.tto_epoch_export_wait(self._h)

    def insert(self, topo, fitness, cell, stream=None):
        _lib.tto_archive_insert(self._h, topo, int(topo.shape[0]), fitness, cell, _stream(stream))

    def propose(self, seed, iteration, B, mutation=DEFAULT_MUTATION, stream=None):
        torch = _torch()
        out = torch.empty(B, self.grid.genome_width, dtype=torch.int32, device=f"cuda:{self.grid.device}")
        _lib.tto_mapelites_propose(self._h, seed, iteration, B, mutation, out, _stream(stream))
        return out

    def step(self, seed, iteration, B, mutation=DEFAULT_MUTATION, precision=PREC_FP32,
             fitness_kind=FIT_WORKLOAD, topo_out=None, fitness_out=None, stream=None):
        o = _lib.EvalOpts(precision, fitness_kind, self.d_split, self.d_moved, self.d_disc)
        _lib.tto_mapelites_step(self._h, seed, iteration, B, mutation, o, topo_out, fitness_out,
                                _stream(stream))

    def step_screened(self, surrogate, seed, iteration, n_propose, n_exact, rank_by=SCREEN_SCORE,
                      mutation=DEFAULT_MUTATION, precision=PREC_FP32, fitness_kind=FIT_WORKLOAD,
                      train_steps=1, topo_out=None, fitness_out=None, score_out=None, stream=None):
        """One surrogate-screened iteration: propose n_propose, evaluate the
        n_exact ranked first exactly, insert, learn from them."""
        o = _lib.EvalOpts(precision, fitness_kind, self.d_split, self.d_moved, self.d_disc)
        _lib.tto_mapelites_step_screened(self._h, surrogate.handle, seed, iteration, n_propose,
                                         n_exact, rank_by, mutation, o, train_steps, topo_out,
                                         fitness_out, score_out, _stream(stream))


class Surrogate:
    """Learned screen of MapElites proposals on one grid: an MLP (three
    hidden ReLU layers) predicting log1p(-fitness) from split-station values
    and post-split loadings, trained online on exact pairs."""

    def __init__(self, grid: Grid, hidden=512, n_load=256, replay=262144, minibatch=8192,
                 lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0):
        _torch()
        self.grid = grid
        self.hidden = hidden
        self.n_load = n_load
        self._h = _lib.tto_surrogate_create(grid.handle, hidden, n_load, replay, minibatch, lr,
                                            beta1, beta2, eps, seed)
        info = _lib.tto_surrogate_info(self._h, n_load)
        self.n_params = info["n_params"]
        self.input_dim = info["input_dim"]
        self.rows = info["rows"]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            _lib.tto_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def replay_fill(self):
        return _lib.tto_surrogate_info(self._h, self.n_load)["replay_fill"]

    def target_stats(self):
        """(mean, deviation) that standardise the training targets."""
        i = _lib.tto_surrogate_info(self._h, self.n_load)
        return i["target_mean"], i["target_std"]

    def params(self, set_values=None):
        """Packed FP32 parameters W1, b1, W2, b2, W3, b3, w4, b4 (numpy)."""
        return _lib.tto_surrogate_params(self._h, self.n_params, set_values)

    def score(self, topo, stream=None):
        torch = _torch()
        topo = topo.contiguous()
        out = torch.empty(int(topo.shape[0]), dtype=torch.float32, device=topo.device)
        _lib.tto_surrogate_score(self._h, topo, int(topo.shape[0]), out, _stream(stream))
        return out

    def features(self, B):
        """(station per slot, eight values per slot, loadings, valid) of the
        last processed batch, as numpy arrays."""
        return _lib.tto_surrogate_features(self._h, B, self.grid.k_max, self.n_load)

    def trace(self, B):
        """Intermediate values of the last batch (first B rows) as numpy
        arrays: h [3][B][H] hidden activations, y [B] raw output, and after
        :meth:`grad` the targets t, output gradient dy and backward signals
        dh [3][B][H]."""
        return _lib.tto_surrogate_trace(self._h, B, self.hidden)

    def add(self, topo, fitness, stream=None):
        _lib.tto_surrogate_add(self._h, topo.contiguous(), int(topo.shape[0]), fitness.contiguous(),
                               _stream(stream))

    def train(self, steps=1, want_loss=True, stream=None):
        return _lib.tto_surrogate_train(self._h, steps, want_loss, _stream(stream))

    def grad(self, topo, fitness, stream=None):
        """(loss, packed gradient) of the mean squared error on one batch of
        exact pairs (targets standardised as in training)."""
        return _lib.tto_surrogate_grad(self._h, topo.contiguous(), int(topo.shape[0]),
                                       fitness.contiguous(), self.n_params, _stream(stream))


def evaluate_multi(jobs, precision=PREC_FP32, fitness_kind=FIT_WORKLOAD, d_split=8, d_moved=8,
                   mode=_lib.MULTI_GRAPH, stream=None):
    """Evaluate several (Grid, topology tensor) pairs as one unit of work.
    jobs: list of (grid, topo) or (grid, topo, timesteps); returns a list of
    output dicts (fitness, desc, cell, island, metrics)."""
    torch = _torch()
    recs, outs = [], []
    for j in jobs:
        g, topo = j[0], j[1].contiguous()
        ts = j[2] if len(j) > 2 else None
        B = int(topo.shape[0])
        if topo.dtype != torch.int32 or not topo.is_cuda or topo.dim() != 2 or topo.shape[1] != g.genome_width:
            raise TTOError(_lib.TTO_E_ARG, "each job's topo must be a CUDA int32 tensor [B][k_max + n_dslot]")
        dev = topo.device
        o = dict(fitness=torch.empty(B, dtype=torch.float32, device=dev),
                 desc=torch.empty(B, 2, dtype=torch.int32, device=dev),
                 cell=torch.empty(B, dtype=torch.int32, device=dev),
                 island=torch.empty(B, dtype=torch.uint8, device=dev),
                 metrics=torch.empty(B, 4, dtype=torch.float32, device=dev))
        outs.append(o)
        recs.append(dict(grid=g.handle, topo=topo, B=B, timesteps=ts, **o))
    _lib.tto_evaluate_multi(recs, _lib.EvalOpts(precision, fitness_kind, d_split, d_moved, 1), mode,
                            _stream(stream))
    return outs


def philox_blocks(seed, iteration, cand, block, n, stream=None):
    torch = _torch()
    out = torch.empty(n, 4, dtype=torch.int32, device="cuda")
    _lib.tto_philox_blocks(seed, iteration, cand, block, n, out, _stream(stream))
    return out
