"""Mixed-grid batching (tto_evaluate_multi), sweep tile variants and the
autotuner, against per-grid evaluation and the FP64 oracle."""
import numpy as np
import pytest

from oracle import dcflow
from synth import config_grid, limits_from_flows, make_grid, random_topologies
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _limited(sg, n_tight=3):
    return sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], n_tight, seed=sg.seed))


def _mixed_grids():
    """Four small grids spanning the timestep passes of the tensor-core sweep
    (T = 1, 4, 16, 24) with ragged batches."""
    specs = [(60, 90, 5, 1, 41), (120, 180, 8, 4, 37), (200, 300, 12, 16, 50), (300, 450, 16, 24, 20)]
    out = []
    for i, (n, e, st, T, B) in enumerate(specs):
        sg = make_grid(n, e, st, assets=(4, 8), T=T, b_dist=("loguniform", 2.0, 200.0),
                       noise=0.1 if T > 1 else 0.0, seed=40 + i, k_max=3, name=f"mixsmall{i}")
        out.append((_limited(sg), B))
    return out


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items() if not k.startswith("_")}


@pytest.mark.parametrize("prec", [0, 3])
def test_multi_equals_per_grid_in_every_mode(prec):
    from paper_2605_10128_b300 import Grid, evaluate_multi, _lib
    grids = []
    for sg, B in _mixed_grids():
        g = Grid(sg)
        topo = torch.tensor(random_topologies(sg, B, seed=B), dtype=torch.int32, device="cuda")
        grids.append((sg, g, topo))
    ref = []
    for sg, g, topo in grids:
        r = g.evaluate(topo, precision=prec, metrics=True)
        g.sync_status()
        ref.append(_np(r))
    modes = [_lib.MULTI_SEQUENTIAL, _lib.MULTI_STREAMS, _lib.MULTI_GRAPH, _lib.MULTI_GRAPH]
    if prec == 0:  # the persistent work list (FP32), eager and recorded (first call records, second replays)
        modes += [_lib.MULTI_PERSISTENT, _lib.MULTI_PERSISTENT_GRAPH, _lib.MULTI_PERSISTENT_GRAPH,
                  _lib.MULTI_PERSISTENT]
    for mode in modes:
        outs = evaluate_multi([(g, topo) for _, g, topo in grids], precision=prec, mode=mode)
        torch.cuda.synchronize()
        for (sg, g, _), o, r in zip(grids, outs, ref):
            g.sync_status()
            o = _np(o)
            for k in ["fitness", "desc", "cell", "island", "metrics"]:
                np.testing.assert_array_equal(o[k], r[k], err_msg=f"mode {mode} {sg.name} {k}")


def test_every_sweep_variant_matches_the_oracle():
    from paper_2605_10128_b300 import Grid
    sg = _limited(config_grid("tto30"), 5)
    topo = random_topologies(sg, 96, seed=13)
    g = Grid(sg)
    idx = list(range(96))
    refs = parity.oracle_eval(sg, topo, idx)
    t = torch.tensor(topo, dtype=torch.int32, device="cuda")
    for prec, shapes, tol in [(0, 2, parity.TOL_FP32), (3, 5, parity.TOL_FP32), (1, 4, parity.TOL_BF16)]:
        for sh in range(shapes):
            g.set_sweep_shape(prec, sh)
            out = _np(g.evaluate(t, precision=prec, metrics=True, fmax=True))
            g.sync_status()
            parity.compare(sg, out, idx, refs, tol=tol)
        g.set_sweep_shape(prec, -1)


def test_autotune_picks_a_variant_and_keeps_results():
    """The mma.sync variants (0-3) share one arithmetic and agree bit for bit;
    the tcgen05 variant (4) sums the TF32 products in the tensor core's order
    and agrees to FP32 rounding; the autotuned evaluation equals the chosen
    variant's exactly."""
    from paper_2605_10128_b300 import Grid
    sg = _limited(config_grid("tto30"), 5)
    g = Grid(sg)
    t = torch.tensor(random_topologies(sg, 128, seed=2), dtype=torch.int32, device="cuda")
    per = []
    for sh in range(5):
        g.set_sweep_shape(3, sh)
        per.append(_np(g.evaluate(t, precision=3, fmax=True)))
    g.set_sweep_shape(3, -1)
    for sh in range(1, 4):
        np.testing.assert_array_equal(per[sh]["fmax"], per[0]["fmax"])
    np.testing.assert_allclose(per[4]["fmax"], per[0]["fmax"], rtol=1e-6, atol=1e-7)
    shape, ms = g.autotune(128, precision=3)
    assert 0 <= shape < 5 and len(ms) == 5 and all(m > 0 for m in ms)
    assert ms[shape] == min(ms)
    tuned = _np(g.evaluate(t, precision=3, fmax=True))
    g.sync_status()
    np.testing.assert_array_equal(tuned["fmax"], per[shape]["fmax"])
    np.testing.assert_array_equal(tuned["cell"], per[shape]["cell"])
    np.testing.assert_array_equal(tuned["fitness"], per[shape]["fitness"])
    s32, ms32 = g.autotune(128, precision=0)
    assert 0 <= s32 < 2 and ms32[s32] == min(ms32[:2])


def test_multi_rejects_bad_jobs():
    from paper_2605_10128_b300 import Grid, TTOError, evaluate_multi
    sg = _limited(config_grid("tto30"), 5)
    g = Grid(sg)
    t = torch.tensor(random_topologies(sg, 8, seed=1), dtype=torch.int32, device="cuda")
    with pytest.raises(TTOError):
        evaluate_multi([(g, t), (g, t)])  # one grid twice


@pytest.mark.parametrize("fitness_kind", [0, 1])
def test_persistent_work_list_mixed_ranks_and_subsets(fitness_kind):
    """The persistent work list over grids of genome rank 2, 3, 6 and 8 (the
    rank-4 and rank-8 bodies), a reordered timestep subset and both fitness
    kinds, equal bit for bit to per-grid evaluation; the tuned FP32 variant of
    a grid does not change the results.  TF32X3 is refused in this mode."""
    from paper_2605_10128_b300 import Grid, TTOError, evaluate_multi, _lib
    specs = [(60, 90, 5, 1, 2, 33), (120, 180, 8, 3, 3, 70), (200, 300, 12, 5, 6, 19), (150, 225, 12, 8, 8, 9)]
    jobs, ref = [], []
    for i, (n, e, st, T, k, B) in enumerate(specs):
        sg = _limited(make_grid(n, e, st, assets=(4, 8), T=T, b_dist=("loguniform", 2.0, 200.0),
                                noise=0.1 if T > 1 else 0.0, seed=60 + i, k_max=k, name=f"rank{k}"))
        g = Grid(sg)
        if i == 1:
            g.set_sweep_shape(0, 1)  # the other FP32 tile variant for the per-grid reference
        topo = torch.tensor(random_topologies(sg, B, seed=3 + i), dtype=torch.int32, device="cuda")
        ts = [2, 0] if T == 3 else None
        jobs.append((g, topo, ts) if ts else (g, topo))
        r = g.evaluate(topo, timesteps=ts, fitness_kind=fitness_kind, metrics=True)
        g.sync_status()
        ref.append(_np(r))
    for mode in [_lib.MULTI_PERSISTENT, _lib.MULTI_PERSISTENT_GRAPH, _lib.MULTI_PERSISTENT_GRAPH]:
        outs = evaluate_multi(jobs, fitness_kind=fitness_kind, mode=mode)
        torch.cuda.synchronize()
        for j, o, r in zip(jobs, outs, ref):
            j[0].sync_status()
            o = _np(o)
            for k in ["fitness", "desc", "cell", "island", "metrics"]:
                np.testing.assert_array_equal(o[k], r[k], err_msg=f"mode {mode} {k}")
    with pytest.raises(TTOError):
        evaluate_multi(jobs, precision=3, mode=_lib.MULTI_PERSISTENT)
