"""Busbar outages (lambda_b) and lambda_f2 on the GPU against the brute-force
oracle: the max over busbar outages per monitored row and timestep within the
loading tolerance, the same islanding counts, lambda_b, and lambda_f2 with the
unsplit reference."""
import numpy as np
import pytest

from oracle import dcflow
from synth import config_grid, limits_from_flows, random_topologies
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _grid(name, n_tight, seed=0, **kw):
    sg = config_grid(name, seed=seed, **kw)
    return sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], n_tight, seed=seed))


def _oracle(sg, topo, idx):
    from tests.parity import n_procs
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(n_procs(), len(idx))) as pool:
        return pool.starmap(dcflow.busbar_outages, [(sg, topo[i]) for i in idx])


def _check(sg, out, idx, refs):
    lim = sg.limit[sg.monitored.astype(np.int64)]
    n_checked = 0
    for i, r in zip(idx, refs):
        if r is None:
            assert np.isnan(out["lambda_b"][i]) and out["n_island"][i] == -1
            continue
        assert out["n_island"][i] == r["n_islanded_busbar"], (i, out["n_island"][i], r["n_islanded_busbar"])
        bm = out["bmax"][i].astype(np.float64)
        err = np.abs(bm - r["bmax"]) / lim[None, :]
        allowed = parity.TOL_FP32 + parity.FLOW_ULPS * np.abs(r["bmax"]) / lim[None, :]
        assert np.all(err <= allowed), (i, float(err.max()), float((err / allowed).max()))
        band = (parity.TOL_FP32 * lim[None, :] + parity.FLOW_ULPS * np.abs(r["bmax"])).sum()
        assert abs(out["lambda_b"][i] - r["lambda_b"]) <= band + 1e-5 * abs(r["lambda_b"]) + 1e-6
        n_checked += 1
    return n_checked


def _run(g, topo):
    out = g.busbar(torch.tensor(topo, dtype=torch.int32, device="cuda"), bmax=True)
    g.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("disc", [False, True])
def test_busbar_outages_tto30(disc):
    from paper_2605_10128_b300 import Grid
    kw = dict(n_disc=12, n_dslot=2) if disc else {}
    sg = _grid("tto30", 5, **kw)
    g = Grid(sg)
    topo = random_topologies(sg, 64, seed=9)
    topo[0] = -1
    idx = list(range(len(topo)))
    refs = _oracle(sg, topo, idx)
    assert _check(sg, _run(g, topo), idx, refs) > 20
    assert any(r is not None and r["n_islanded_busbar"] > 0 for r in refs)


def test_busbar_outages_tto2k_sampled():
    from paper_2605_10128_b300 import Grid
    sg = _grid("tto2k", 30)
    g = Grid(sg)
    topo = random_topologies(sg, 32, seed=10)
    idx = [0, 1, 2]
    assert _check(sg, _run(g, topo), idx, _oracle(sg, topo, idx)) >= 1


@pytest.mark.parametrize("mode", ["fp32", "tcgen05", "mma"])
def test_lambda_f2_fitness(mode):
    """lambda_f2 with the N-1 sweep in FP32, on the tcgen05 kernel (whose
    operand layouts the split update writes, plain U rows kept for the busbar
    sweep) and on an mma.sync variant."""
    from paper_2605_10128_b300 import Grid, TTOError, FIT_F2, PREC_FP32, PREC_TF32X3
    sg = _grid("tto30", 5)
    g = Grid(sg)
    prec = PREC_FP32 if mode == "fp32" else PREC_TF32X3
    if mode != "fp32":
        g.set_sweep_shape(PREC_TF32X3, 4 if mode == "tcgen05" else 0)
    topo = random_topologies(sg, 48, seed=11)
    t = torch.tensor(topo, dtype=torch.int32, device="cuda")
    with pytest.raises(TTOError):
        g.evaluate(t, fitness_kind=FIT_F2, precision=prec)
    g.busbar_reference()
    g.profile(True)
    out = g.evaluate(t, fitness_kind=FIT_F2, metrics=True, fmax=True, precision=prec)
    g.evaluate(t, precision=prec)  # a plain evaluation: no busbar stage
    stage, n_calls = g.profile_read()
    g.profile(False)
    assert n_calls == 2 and min(stage[:3]) > 0 and stage[3] > 0  # split, N-1 sweep, metrics, busbar sweep
    g.sync_status()
    out = {k: v.cpu().numpy() for k, v in out.items() if not k.startswith("_")}
    idx = list(range(len(topo)))
    ev = parity.oracle_eval(sg, topo, idx)
    bb = _oracle(sg, topo, idx)
    pre = dcflow.busbar_outages(sg, np.full(sg.genome_width, -1))["lambda_b"]
    lim = sg.limit[sg.monitored.astype(np.int64)]
    for i, (r, b) in enumerate(zip(ev, bb)):
        if r["island_base"]:
            assert out["fitness"][i] == -np.inf
            continue
        ref = dcflow.lambda_f2(r, b, pre)
        band = (parity.TOL_FP32 * lim[None, :] + parity.FLOW_ULPS * np.abs(r["fmax"])).sum()
        bandb = (parity.TOL_FP32 * lim[None, :] + parity.FLOW_ULPS * np.abs(b["bmax"])).sum()
        near = int((np.abs(r["fmax"] - lim[None, :]) <= parity.TOL_FP32 * lim[None, :]).sum())
        near0 = int((np.abs(np.abs(r["fprime"]) - lim[None, :]) <= parity.TOL_FP32 * lim[None, :]).sum())
        bound = band + bandb + 50.0 * near + 200.0 * near0 + 1e-5 * abs(ref) + 1e-6
        assert abs(out["fitness"][i] - ref) <= bound, (i, out["fitness"][i], ref)
    # changing the limits drops the reference
    g.set_limits(sg.limit * 1.01)
    with pytest.raises(TTOError):
        g.evaluate(t, fitness_kind=FIT_F2, precision=prec)


@pytest.mark.parametrize("T", [2, 5, 24, 32])
def test_busbar_outages_every_timestep_shape(T):
    """Timestep counts that pad to 2, 8 (5 real), 24 and 32: the kernels that
    take two rows per thread, with paired bmax stores, and the one-row kernels
    of long horizons."""
    from paper_2605_10128_b300 import Grid
    from synth import make_grid
    sg = make_grid(120, 180, 10, assets=(4, 8), T=T, b_dist=("loguniform", 2.0, 200.0), noise=0.1,
                   seed=40 + T, k_max=4, name="busbar_T")
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 3, seed=T))
    g = Grid(sg)
    topo = random_topologies(sg, 24, seed=T)
    idx = list(range(len(topo)))
    assert _check(sg, _run(g, topo), idx, _oracle(sg, topo, idx)) > 10


def test_busbar_timestep_subset_and_empty_batch():
    """A reordered subset of the timesteps (3 of 24, padded to 4) against the
    oracle on the same subset, and an empty batch."""
    from paper_2605_10128_b300 import Grid
    from synth import make_grid
    sg = make_grid(120, 180, 10, assets=(4, 8), T=24, b_dist=("loguniform", 2.0, 200.0), noise=0.1,
                   seed=64, k_max=4, name="busbar_T")
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 3, seed=1))
    g = Grid(sg)
    topo = random_topologies(sg, 24, seed=3)
    ts = [23, 0, 7]
    out = g.busbar(torch.tensor(topo, dtype=torch.int32, device="cuda"), timesteps=ts, bmax=True)
    g.sync_status()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    assert out["bmax"].shape == (24, 3, len(sg.monitored))
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(parity.n_procs(), 8)) as pool:
        refs = pool.starmap(dcflow.busbar_outages, [(sg, topo[i], ts) for i in range(24)])
    assert _check(sg, out, list(range(24)), refs) > 10
    empty = g.busbar(torch.empty((0, sg.genome_width), dtype=torch.int32, device="cuda"), bmax=True)
    g.sync_status()
    assert empty["lambda_b"].shape == (0,) and empty["bmax"].shape == (0, sg.T, len(sg.monitored))
