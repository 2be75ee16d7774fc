"""ctypes binding of libtto.so: one Python function per C entry point, same
names, argument marshalling only (every step of the computation runs in the
library's CUDA kernels).  Device buffers are torch CUDA tensors; their
addresses are passed as plain pointers together with the current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtto.so")

TTO_OK = 0
TTO_E_ARG = -1
TTO_E_DISCONNECTED = -2
TTO_E_CUDA = -3
TTO_E_NOMEM = -4
TTO_E_TOPOLOGY = -5
TTO_E_TIMEOUT = -6
PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_TF32X3, PREC_FP16X3 = 0, 1, 2, 3, 4
FIT_WORKLOAD, FIT_F1, FIT_F2 = 0, 1, 2

_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)
_f64p = C.POINTER(C.c_double)
_vp = C.c_void_p


class TTOError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tto error {code}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("from_", _i32p), ("to", _i32p),
                ("b", _f64p), ("slack", C.c_int32), ("n_time", C.c_int32), ("p", _f64p),
                ("limit", _f64p), ("n_monitored", C.c_int32), ("monitored", _i32p),
                ("n_outage", C.c_int32), ("outage", _i32p), ("n_station", C.c_int32),
                ("station_bus", _i32p), ("asset_offset", _i32p), ("asset_branch", _i32p),
                ("n_action", C.c_int32), ("action_station", _i32p), ("action_mask", _u32p),
                ("k_max", C.c_int32), ("device", C.c_int32), ("n_disc", C.c_int32),
                ("disc_branch", _i32p), ("n_dslot", C.c_int32)]


class EvalOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("fitness_kind", C.c_int32), ("d_split", C.c_int32),
                ("d_moved", C.c_int32), ("d_disc", C.c_int32)]


class EvalJob(C.Structure):
    _fields_ = [("grid", _vp), ("topo", _vp), ("B", C.c_int32), ("timesteps", _i32p), ("n_t", C.c_int32),
                ("fitness", _vp), ("desc", _vp), ("cell", _vp), ("island", _vp), ("metrics", _vp)]


MULTI_SEQUENTIAL, MULTI_STREAMS, MULTI_GRAPH, MULTI_PERSISTENT, MULTI_PERSISTENT_GRAPH = 0, 1, 2, 3, 4
SCREEN_SCORE, SCREEN_CELL_GAIN = 0, 1


class MutParams(C.Structure):
    _fields_ = [("p_add", C.c_double), ("p_remove", C.c_double), ("p_change", C.c_double),
                ("p_identity", C.c_double), ("n_mut_mean", C.c_double), ("dp_add", C.c_double),
                ("dp_remove", C.c_double), ("dp_change", C.c_double), ("dp_identity", C.c_double),
                ("crossover", C.c_int32), ("p_c1", C.c_double)]


# Algorithm 1's disconnection-operation probabilities (add, remove, change,
# identity) and Algorithm 2's default bias when a caller gives none.
DEFAULT_DISC_PROBS = (0.25, 0.25, 0.5, 0.0)
DEFAULT_P_C1 = 0.5


class SurrogateCfg(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("n_load", C.c_int32), ("replay", C.c_int32),
                ("minibatch", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64)]


_lib = None

_SIGS = {
    "tto_grid_create": ([C.POINTER(GridDesc), C.POINTER(_vp)], C.c_int),
    "tto_grid_destroy": ([_vp], C.c_int),
    "tto_grid_info": ([_vp, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p], C.c_int),
    "tto_grid_base_flows": ([_vp, _f64p], C.c_int),
    "tto_grid_set_limits": ([_vp, _f64p], C.c_int),
    "tto_grid_reserve": ([_vp, C.c_int32, C.c_int32], C.c_int),
    "tto_evaluate_batch": ([_vp, _vp, C.c_int32, _i32p, C.c_int32, C.POINTER(EvalOpts), _vp, _vp,
                            _vp, _vp, _vp, _vp, _vp], C.c_int),
    "tto_evaluate_batch_static": ([_vp, _vp, C.c_int32, _i32p, C.c_int32, C.POINTER(EvalOpts), _vp,
                                   _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "tto_grid_sync_status": ([_vp, _vp], C.c_int),
    "tto_debug_bounded_wait": ([_vp, C.c_int64, _vp], C.c_int),
    "tto_grid_autotune": ([_vp, C.c_int32, C.c_int32, C.c_int32, _i32p, C.POINTER(C.c_float), _vp], C.c_int),
    "tto_grid_set_sweep_shape": ([_vp, C.c_int32, C.c_int32], C.c_int),
    "tto_evaluate_multi": ([C.POINTER(EvalJob), C.c_int32, C.POINTER(EvalOpts), C.c_int32, _vp], C.c_int),
    "tto_grid_profile": ([_vp, C.c_int32], C.c_int),
    "tto_grid_profile_read": ([_vp, C.POINTER(C.c_float), _i32p], C.c_int),
    "tto_archive_create": ([_vp, C.c_int32, C.c_int32, C.POINTER(_vp)], C.c_int),
    "tto_archive_create_ex": ([_vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(_vp)], C.c_int),
    "tto_grid_disc_info": ([_vp, _i32p, _i32p], C.c_int),
    "tto_worst_k": ([_vp, _vp, C.c_int32, _i32p, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "tto_epoch_export": ([_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "tto_epoch_export_wait": ([_vp], C.c_int),
    "tto_evaluate_busbar": ([_vp, _vp, C.c_int32, _i32p, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "tto_grid_busbar_reference": ([_vp, _i32p, C.c_int32, _vp], C.c_int),
    "tto_archive_destroy": ([_vp], C.c_int),
    "tto_archive_export": ([_vp, _vp, _vp, _vp], C.c_int),
    "tto_archive_import": ([_vp, _vp, _vp, _vp], C.c_int),
    "tto_archive_insert": ([_vp, _vp, C.c_int32, _vp, _vp, _vp], C.c_int),
    "tto_mapelites_propose": ([_vp, C.c_uint64, C.c_uint64, C.c_int32, C.POINTER(MutParams), _vp,
                               _vp], C.c_int),
    "tto_mapelites_step": ([_vp, C.c_uint64, C.c_uint64, C.c_int32, C.POINTER(MutParams),
                            C.POINTER(EvalOpts), _vp, _vp, _vp], C.c_int),
    "tto_philox_blocks": ([C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32, _vp, _vp],
                          C.c_int),
    "tto_surrogate_create": ([_vp, C.POINTER(SurrogateCfg), C.POINTER(_vp)], C.c_int),
    "tto_surrogate_destroy": ([_vp], C.c_int),
    "tto_surrogate_info": ([_vp, C.POINTER(C.c_int64), _i32p, _i32p, _vp, _vp], C.c_int),
    "tto_surrogate_params": ([_vp, _vp, _vp], C.c_int),
    "tto_surrogate_score": ([_vp, _vp, C.c_int32, _vp, _vp], C.c_int),
    "tto_surrogate_features": ([_vp, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "tto_surrogate_trace": ([_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "tto_surrogate_add": ([_vp, _vp, C.c_int32, _vp, _vp], C.c_int),
    "tto_surrogate_train": ([_vp, C.c_int32, C.POINTER(C.c_float), _vp], C.c_int),
    "tto_surrogate_grad": ([_vp, _vp, C.c_int32, _vp, C.POINTER(C.c_float), _vp, _vp], C.c_int),
    "tto_mapelites_step_screened": ([_vp, _vp, C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, C.c_int32,
                                     C.POINTER(MutParams), C.POINTER(EvalOpts), C.c_int32, _vp, _vp,
                                     _vp, _vp], C.c_int),
    "tto_last_error": ([], C.c_char_p),
}


def lib():
    """The loaded library; raises if it has not been built (there is no
    fallback implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2605_10128_b300.build`")
        h = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(h, name)
            fn.argtypes = args
            fn.restype = res
        _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


def check(rc):
    if rc != TTO_OK:
        raise TTOError(rc, lib().tto_last_error().decode())
    return rc


def _ptr(arr, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


def tto_grid_create(grid, device=0):
    """Create a library grid from an object with the fields of a grid
    description (see synth.SynthGrid); returns (handle, keepalive)."""
    keep = dict(
        fr=np.ascontiguousarray(grid.from_bus, dtype=np.int32),
        to=np.ascontiguousarray(grid.to_bus, dtype=np.int32),
        b=np.ascontiguousarray(grid.b, dtype=np.float64),
        p=np.ascontiguousarray(grid.p, dtype=np.float64),
        lim=np.ascontiguousarray(grid.limit if grid.limit is not None else np.ones(len(grid.b)),
                                 dtype=np.float64),
        mon=np.ascontiguousarray(grid.monitored, dtype=np.int32),
        out=np.ascontiguousarray(grid.outages, dtype=np.int32),
        sb=np.ascontiguousarray(grid.station_bus, dtype=np.int32),
        ao=np.ascontiguousarray(grid.asset_offset, dtype=np.int32),
        ab=np.ascontiguousarray(grid.asset_branch, dtype=np.int32),
        ast=np.ascontiguousarray(grid.action_station, dtype=np.int32),
        am=np.ascontiguousarray(grid.action_mask, dtype=np.uint32),
        disc=np.ascontiguousarray(getattr(grid, "disc", np.zeros(0)), dtype=np.int32),
    )
    d = GridDesc()
    d.n_bus = int(grid.n_bus)
    d.n_branch = int(keep["fr"].size)
    d.from_ = _ptr(keep["fr"], C.c_int32)
    d.to = _ptr(keep["to"], C.c_int32)
    d.b = _ptr(keep["b"], C.c_double)
    d.slack = int(grid.slack)
    d.n_time = int(keep["p"].shape[0])
    d.p = _ptr(keep["p"], C.c_double)
    d.limit = _ptr(keep["lim"], C.c_double)
    d.n_monitored = int(keep["mon"].size)
    d.monitored = _ptr(keep["mon"], C.c_int32)
    d.n_outage = int(keep["out"].size)
    d.outage = _ptr(keep["out"], C.c_int32)
    d.n_station = int(keep["sb"].size)
    d.station_bus = _ptr(keep["sb"], C.c_int32)
    d.asset_offset = _ptr(keep["ao"], C.c_int32)
    d.asset_branch = _ptr(keep["ab"], C.c_int32)
    d.n_action = int(keep["ast"].size)
    d.action_station = _ptr(keep["ast"], C.c_int32)
    d.action_mask = _ptr(keep["am"], C.c_uint32)
    d.k_max = int(grid.k_max)
    d.device = int(device)
    d.n_disc = int(keep["disc"].size)
    d.disc_branch = _ptr(keep["disc"], C.c_int32) if keep["disc"].size else None
    d.n_dslot = int(getattr(grid, "n_dslot", 0))
    h = _vp()
    check(lib().tto_grid_create(C.byref(d), C.byref(h)))
    return h


def tto_grid_destroy(h):
    return check(lib().tto_grid_destroy(h))


def tto_grid_info(h):
    v = [C.c_int32() for _ in range(6)]
    check(lib().tto_grid_info(h, *[C.byref(x) for x in v]))
    keys = ["n_branch", "n_monitored", "n_outage", "n_time", "k_max", "n_action"]
    return {k: x.value for k, x in zip(keys, v)}


def tto_worst_k(h, topo, n, timesteps, k, outage_out, energy_out, all_energy, stream):
    ts = None
    n_t = 0
    if timesteps is not None:
        ts_arr = np.ascontiguousarray(timesteps, dtype=np.int32)
        ts = _ptr(ts_arr, C.c_int32)
        n_t = int(ts_arr.size)
    return check(lib().tto_worst_k(h, _dp(topo), int(n), ts, n_t, int(k), _dp(outage_out), _dp(energy_out),
                                   _dp(all_energy), _vp(stream)))


def _ts(timesteps):
    if timesteps is None:
        return None, 0, None
    ts_arr = np.ascontiguousarray(timesteps, dtype=np.int32)
    return _ptr(ts_arr, C.c_int32), int(ts_arr.size), ts_arr


def tto_evaluate_busbar(h, topo, B, timesteps, lambda_b, n_island, bmax, stream):
    ts, n_t, keep = _ts(timesteps)
    return check(lib().tto_evaluate_busbar(h, _dp(topo), int(B), ts, n_t, _dp(lambda_b), _dp(n_island), _dp(bmax),
                                           _vp(stream)))


def tto_grid_busbar_reference(h, timesteps, stream):
    ts, n_t, keep = _ts(timesteps)
    return check(lib().tto_grid_busbar_reference(h, ts, n_t, _vp(stream)))


def tto_epoch_export(a, k, fit, gen, filled, widx, wval, stream):
    return check(lib().tto_epoch_export(a, int(k), _dp(fit), _dp(gen), _dp(filled), _dp(widx), _dp(wval),
                                        _vp(stream)))


def tto_epoch_export_wait(a):
    return check(lib().tto_epoch_export_wait(a))


def tto_grid_disc_info(h):
    nd, ns = C.c_int32(), C.c_int32()
    check(lib().tto_grid_disc_info(h, C.byref(nd), C.byref(ns)))
    return nd.value, ns.value


def tto_grid_base_flows(h, n_time, n_branch):
    f0 = np.zeros((n_time, n_branch), dtype=np.float64)
    check(lib().tto_grid_base_flows(h, _ptr(f0, C.c_double)))
    return f0


def tto_grid_set_limits(h, limit):
    lim = np.ascontiguousarray(limit, dtype=np.float64)
    return check(lib().tto_grid_set_limits(h, _ptr(lim, C.c_double)))


def tto_grid_reserve(h, max_batch, n_t):
    return check(lib().tto_grid_reserve(h, int(max_batch), int(n_t)))


def _dp(t):
    return None if t is None else _vp(t.data_ptr())


def tto_evaluate_batch(h, topo, B, timesteps, opts, fitness, desc, cell, island, metrics, fmax,
                       stream):
    ts = None
    n_t = 0
    if timesteps is not None:
        ts_arr = np.ascontiguousarray(timesteps, dtype=np.int32)
        ts = _ptr(ts_arr, C.c_int32)
        n_t = int(ts_arr.size)
    return check(lib().tto_evaluate_batch(h, _dp(topo), int(B), ts, n_t, C.byref(opts),
                                          _dp(fitness), _dp(desc), _dp(cell), _dp(island),
                                          _dp(metrics), _dp(fmax), _vp(stream)))


def tto_evaluate_batch_static(h, topo, B, timesteps, opts, fitness, desc, cell, island, metrics,
                              fmax, stream):
    """The allocation-free evaluation entry point (library-owned fixed scratch)."""
    ts = None
    n_t = 0
    if timesteps is not None:
        ts_arr = np.ascontiguousarray(timesteps, dtype=np.int32)
        ts = _ptr(ts_arr, C.c_int32)
        n_t = int(ts_arr.size)
    return check(lib().tto_evaluate_batch_static(h, _dp(topo), int(B), ts, n_t, C.byref(opts),
                                                 _dp(fitness), _dp(desc), _dp(cell), _dp(island),
                                                 _dp(metrics), _dp(fmax), _vp(stream)))


def tto_grid_autotune(h, B, n_t, precision, stream):
    shape = C.c_int32()
    ms = (C.c_float * 8)()
    check(lib().tto_grid_autotune(h, int(B), int(n_t), int(precision), C.byref(shape), ms, _vp(stream)))
    return shape.value, list(ms)[:_n_shapes(precision)]


def _n_shapes(precision):
    """Sweep tile variants per precision mode (see tto_grid_autotune)."""
    return 2 if precision == PREC_FP32 else (5 if precision == PREC_TF32X3 else 4)


def tto_grid_set_sweep_shape(h, precision, shape):
    return check(lib().tto_grid_set_sweep_shape(h, int(precision), int(shape)))


def tto_evaluate_multi(jobs, opts, mode, stream):
    """jobs: list of dicts with grid (handle), topo, B, timesteps (or None),
    fitness, desc, cell, island, metrics (tensors or None)."""
    arr = (EvalJob * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        e = arr[i]
        e.grid = j["grid"]
        e.topo = _dp(j["topo"])
        e.B = int(j["B"])
        if j.get("timesteps") is not None:
            ts = np.ascontiguousarray(j["timesteps"], dtype=np.int32)
            keep.append(ts)
            e.timesteps = _ptr(ts, C.c_int32)
            e.n_t = int(ts.size)
        else:
            e.timesteps = None
            e.n_t = 0
        for f in ("fitness", "desc", "cell", "island", "metrics"):
            setattr(e, f, _dp(j.get(f)))
    return check(lib().tto_evaluate_multi(arr, len(jobs), C.byref(opts), int(mode), _vp(stream)))


def tto_debug_bounded_wait(h, cycles, stream):
    return check(lib().tto_debug_bounded_wait(h, int(cycles), _vp(stream)))


def tto_grid_sync_status(h, stream):
    return check(lib().tto_grid_sync_status(h, _vp(stream)))


def tto_grid_profile(h, enable):
    return check(lib().tto_grid_profile(h, int(enable)))


def tto_grid_profile_read(h):
    ms = (C.c_float * 4)()
    n = C.c_int32()
    check(lib().tto_grid_profile_read(h, ms, C.byref(n)))
    return [ms[0], ms[1], ms[2], ms[3]], n.value


def tto_archive_create(grid_h, d_split, d_moved, d_disc=1):
    a = _vp()
    if d_disc == 1:
        check(lib().tto_archive_create(grid_h, int(d_split), int(d_moved), C.byref(a)))
    else:
        check(lib().tto_archive_create_ex(grid_h, int(d_split), int(d_moved), int(d_disc), C.byref(a)))
    return a


def tto_archive_destroy(a):
    return check(lib().tto_archive_destroy(a))


def tto_archive_export(a, cells, k_max):
    fit = np.zeros(cells, dtype=np.float32)
    gen = np.zeros((cells, k_max), dtype=np.int32)
    filled = np.zeros(cells, dtype=np.uint8)
    check(lib().tto_archive_export(a, fit.ctypes.data, gen.ctypes.data, filled.ctypes.data))
    return fit, gen, filled


def tto_archive_import(a, fit, gen, filled):
    fit = np.ascontiguousarray(fit, dtype=np.float32)
    gen = np.ascontiguousarray(gen, dtype=np.int32)
    filled = np.ascontiguousarray(filled, dtype=np.uint8)
    return check(lib().tto_archive_import(a, fit.ctypes.data, gen.ctypes.data, filled.ctypes.data))


def tto_archive_insert(a, topo, B, fitness, cell, stream):
    return check(lib().tto_archive_insert(a, _dp(topo), int(B), _dp(fitness), _dp(cell),
                                          _vp(stream)))


def _mut(mp):
    """MutParams from (p_add, p_remove, p_change, p_identity, n_mut_mean[,
    dp_add, dp_remove, dp_change, dp_identity[, crossover, p_c1]])."""
    m = MutParams()
    m.p_add, m.p_remove, m.p_change, m.p_identity = mp[0], mp[1], mp[2], mp[3]
    m.n_mut_mean = mp[4]
    dp = tuple(mp[5:9]) if len(mp) >= 9 else DEFAULT_DISC_PROBS
    m.dp_add, m.dp_remove, m.dp_change, m.dp_identity = dp
    m.crossover = int(mp[9]) if len(mp) >= 10 else 0
    m.p_c1 = float(mp[10]) if len(mp) >= 11 else DEFAULT_P_C1
    return m


def tto_mapelites_propose(a, seed, iteration, B, mut, topo_out, stream):
    m = _mut(mut)
    return check(lib().tto_mapelites_propose(a, int(seed), int(iteration), int(B), C.byref(m),
                                             _dp(topo_out), _vp(stream)))


def tto_mapelites_step(a, seed, iteration, B, mut, opts, topo_out, fitness_out, stream):
    m = _mut(mut)
    return check(lib().tto_mapelites_step(a, int(seed), int(iteration), int(B), C.byref(m),
                                          C.byref(opts), _dp(topo_out), _dp(fitness_out),
                                          _vp(stream)))


def tto_philox_blocks(seed, iteration, cand, block, n, out, stream):
    return check(lib().tto_philox_blocks(int(seed), int(iteration), int(cand), int(block), int(n),
                                         _dp(out), _vp(stream)))


def tto_surrogate_create(grid_h, hidden, n_load, replay, minibatch, lr, beta1, beta2, eps, seed):
    cfg = SurrogateCfg(int(hidden), int(n_load), int(replay), int(minibatch), float(lr), float(beta1),
                       float(beta2), float(eps), int(seed))
    h = _vp()
    check(lib().tto_surrogate_create(grid_h, C.byref(cfg), C.byref(h)))
    return h


def tto_surrogate_destroy(h):
    return check(lib().tto_surrogate_destroy(h))


def tto_surrogate_info(h, n_load):
    n = C.c_int64()
    d = C.c_int32()
    fill = C.c_int32()
    rows = np.zeros(n_load, dtype=np.int32)
    stats = np.zeros(2, dtype=np.float32)
    check(lib().tto_surrogate_info(h, C.byref(n), C.byref(d), C.byref(fill), rows.ctypes.data,
                                   stats.ctypes.data))
    return dict(n_params=n.value, input_dim=d.value, replay_fill=fill.value, rows=rows,
                target_mean=float(stats[0]), target_std=float(stats[1]))


def tto_surrogate_params(h, n_params, set_values=None):
    """Returns the packed FP32 parameters (after setting them, if given)."""
    out = np.zeros(n_params, dtype=np.float32)
    src = None
    if set_values is not None:
        src = np.ascontiguousarray(set_values, dtype=np.float32)
        if src.size != n_params:
            raise TTOError(TTO_E_ARG, f"expected {n_params} parameters, got {src.size}")
    check(lib().tto_surrogate_params(h, out.ctypes.data, None if src is None else src.ctypes.data))
    return out


def tto_surrogate_score(h, topo, B, score, stream):
    return check(lib().tto_surrogate_score(h, _dp(topo), int(B), _dp(score), _vp(stream)))


def tto_surrogate_features(h, B, k_max, n_load):
    si = np.zeros((B, k_max), dtype=np.int32)
    sf = np.zeros((B, k_max, 8), dtype=np.float32)
    xd = np.zeros((B, n_load), dtype=np.float32)
    valid = np.zeros(B, dtype=np.int32)
    check(lib().tto_surrogate_features(h, int(B), si.ctypes.data, sf.ctypes.data, xd.ctypes.data,
                                       valid.ctypes.data))
    return si, sf, xd, valid


def tto_surrogate_trace(h, B, hidden):
    hs = np.zeros((3, B, hidden), dtype=np.float32)
    dh = np.zeros((3, B, hidden), dtype=np.float32)
    y = np.zeros(B, dtype=np.float32)
    t = np.zeros(B, dtype=np.float32)
    dy = np.zeros(B, dtype=np.float32)
    check(lib().tto_surrogate_trace(h, int(B), hs.ctypes.data, y.ctypes.data, t.ctypes.data, dy.ctypes.data,
                                    dh.ctypes.data))
    return dict(h=hs, y=y, t=t, dy=dy, dh=dh)


def tto_surrogate_add(h, topo, B, fitness, stream):
    return check(lib().tto_surrogate_add(h, _dp(topo), int(B), _dp(fitness), _vp(stream)))


def tto_surrogate_train(h, steps, want_loss, stream):
    loss = C.c_float()
    check(lib().tto_surrogate_train(h, int(steps), C.byref(loss) if want_loss else None,
                                    _vp(stream)))
    return loss.value if want_loss else None


def tto_surrogate_grad(h, topo, B, fitness, n_params, stream):
    loss = C.c_float()
    grad = np.zeros(n_params, dtype=np.float32)
    check(lib().tto_surrogate_grad(h, _dp(topo), int(B), _dp(fitness), C.byref(loss),
                                   grad.ctypes.data, _vp(stream)))
    return loss.value, grad


def tto_mapelites_step_screened(a, s, seed, iteration, n_propose, n_exact, rank_by, mut, opts,
                                train_steps, topo_out, fitness_out, score_out, stream):
    m = _mut(mut)
    return check(lib().tto_mapelites_step_screened(a, s, int(seed), int(iteration), int(n_propose),
                                                   int(n_exact), int(rank_by), C.byref(m), C.byref(opts),
                                                   int(train_steps), _dp(topo_out), _dp(fitness_out),
                                                   _dp(score_out), _vp(stream)))


def tto_last_error():
    return lib().tto_last_error().decode()
