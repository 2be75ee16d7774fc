"""Worst-k N-1 export (Sec. "AC-Validator") on the GPU against the oracle:
every outage's overload energy within the loading tolerance, the same
islanded/opened exclusions, and a worst-k list that the oracle's energies
confirm up to near-ties."""
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


def _energies(sg, topo, idx):
    res = dcflow.evaluate_many(sg, [topo[i] for i in idx], processes=min(parity.n_procs(), len(idx)),
                               want_energy=True)
    return [np.full(sg.outages.size, np.nan) if r["island_base"] else r["outage_energy"] for r in res]


def _check(sg, out, idx, refs, k):
    lim = sg.limit[sg.monitored.astype(np.int64)]
    bound0 = parity.TOL_FP32 * float(lim.sum()) * sg.T
    for row, (i, E) in enumerate(zip(idx, refs)):
        got = out["all_energy"][i].astype(np.float64)
        assert np.array_equal(np.isnan(got), np.isnan(E)), f"exclusions differ at {i}"
        ok = ~np.isnan(E)
        bound = bound0 + 1e-5 * np.abs(E[ok])
        assert np.all(np.abs(got[ok] - E[ok]) <= bound), (i, float(np.max(np.abs(got[ok] - E[ok]))))
        sel = out["outage"][i]
        val = out["energy"][i]
        n_ok = int(ok.sum())
        assert int((sel >= 0).sum()) == min(k, n_ok)
        assert np.all(sel[min(k, n_ok):] == -1) and np.isnan(val[min(k, n_ok):]).all()
        ref_idx, ref_val = dcflow.worst_k(E, k)
        if n_ok == 0:
            continue
        kth = np.nanmin(ref_val)
        for r_, c in enumerate(sel[: min(k, n_ok)]):
            assert E[c] >= kth - 2 * (bound0 + 1e-5 * abs(kth)), (i, r_, c, E[c], kth)
            assert val[r_] == np.float32(got[c])
        # the GPU's list is in its own energy order
        v = val[: min(k, n_ok)]
        assert np.all(np.diff(v) <= 0)


def test_worst_k_tto30_with_disconnections():
    from paper_2605_10128_b300 import Grid
    sg = _grid("tto30", 5, n_disc=12, n_dslot=2)
    g = Grid(sg)
    topo = random_topologies(sg, 48, seed=6)
    topo[0] = -1  # the unchanged topology
    out = g.worst_k(torch.tensor(topo, dtype=torch.int32, device="cuda"), k=20, all_energy=True)
    g.sync_status()
    out = {k_: v.cpu().numpy() for k_, v in out.items()}
    idx = list(range(len(topo)))
    refs = _energies(sg, topo, idx)
    assert any(np.isnan(E).all() for E in refs)  # some topologies island the grid
    _check(sg, out, idx, refs, 20)


def test_worst_k_tto2k_sampled():
    from paper_2605_10128_b300 import Grid
    sg = _grid("tto2k", 30)
    g = Grid(sg)
    topo = random_topologies(sg, 64, seed=12)
    out = g.worst_k(torch.tensor(topo, dtype=torch.int32, device="cuda"), k=20, all_energy=True)
    g.sync_status()
    out = {k_: v.cpu().numpy() for k_, v in out.items()}
    idx = [0, 1, 2]
    _check(sg, out, idx, _energies(sg, topo, idx), 20)


@pytest.mark.parametrize("T", [2, 5, 24, 32])
def test_worst_k_every_timestep_shape(T):
    """Timestep counts that pad to 2, 8 (5 real), 24 and 32 in the energy
    kernel, whose row loop is unrolled."""
    from paper_2605_10128_b300 import Grid
    from synth import make_grid
    sg = make_grid(120, 180, 10, assets=(4, 8), T=T, b_dist=("loguniform", 2.0, 200.0), noise=0.1,
                   seed=50 + T, k_max=4, name="worstk_T")
    sg = sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 3, seed=T))
    g = Grid(sg)
    topo = random_topologies(sg, 24, seed=T)
    out = g.worst_k(torch.tensor(topo, dtype=torch.int32, device="cuda"), k=20, all_energy=True)
    g.sync_status()
    out = {k_: v.cpu().numpy() for k_, v in out.items()}
    idx = list(range(len(topo)))
    _check(sg, out, idx, _energies(sg, topo, idx), 20)


def test_worst_k_validation_and_large_k():
    from paper_2605_10128_b300 import Grid, TTOError
    sg = _grid("tto30", 5)
    g = Grid(sg)
    t = torch.tensor(random_topologies(sg, 4, seed=1), dtype=torch.int32, device="cuda")
    with pytest.raises(TTOError):
        g.worst_k(t, k=0)
    out = g.worst_k(t, k=200, all_energy=True)  # more than the 41 outages
    g.sync_status()
    sel = out["outage"].cpu().numpy()
    E = out["all_energy"].cpu().numpy()
    for i in range(4):
        n_ok = int((~np.isnan(E[i])).sum())
        assert sorted(sel[i][:n_ok].tolist()) == sorted(np.flatnonzero(~np.isnan(E[i])).tolist())
        assert np.all(sel[i][n_ok:] == -1)


def test_epoch_export_snapshot_and_overlap():
    """The end-of-epoch hand-over: the host copy equals the archive at the
    export point although later iterations were queued behind it, its worst-k
    lists equal tto_worst_k on the exported genomes, and a second export
    orders itself after the first copy."""
    from paper_2605_10128_b300 import Grid, Archive
    sg = _grid("tto2k", 30)  # large enough that the archive keeps improving
    g = Grid(sg)
    A = Archive(g, 8, 8)
    for it in range(3):
        A.step(3, it, 512)
    torch.cuda.synchronize()
    ref_f, ref_g, ref_fl = A.export()
    out = A.epoch_export(k=10)
    for it in range(3, 6):
        A.step(3, it, 512)
    A.epoch_wait()
    g.sync_status()
    np.testing.assert_array_equal(out["fitness"].numpy(), ref_f)
    np.testing.assert_array_equal(out["genome"].numpy(), ref_g)
    np.testing.assert_array_equal(out["filled"].numpy(), ref_fl)
    wk = g.worst_k(torch.tensor(ref_g, dtype=torch.int32, device="cuda"), k=10)
    full = ref_fl.astype(bool)
    assert full.sum() > 5
    np.testing.assert_array_equal(out["worst_outage"].numpy()[full], wk["outage"].cpu().numpy()[full])
    np.testing.assert_array_equal(out["worst_energy"].numpy()[full], wk["energy"].cpu().numpy()[full])
    assert np.all(out["worst_outage"].numpy()[~full] == -1)  # empty cells are skipped
    assert np.isnan(out["worst_energy"].numpy()[~full]).all()
    f_now, g_now, fl_now = A.export()
    assert not np.array_equal(f_now, ref_f)  # the later iterations moved on
    out2 = A.epoch_export(k=10)
    A.epoch_wait()
    np.testing.assert_array_equal(out2["fitness"].numpy(), f_now)
    np.testing.assert_array_equal(out2["genome"].numpy(), g_now)


@pytest.mark.slow
def test_tto10k_full_batch_worst_k_and_busbar_sampled():
    """The 10000-bus workload in the benchmark's batch (8192 topologies): the
    worst-20 export and the busbar outages of the whole batch on the GPU, one
    non-islanded topology re-solved by the oracle over every outage and every
    busbar node."""
    from paper_2605_10128_b300 import Grid
    from synth import CONFIGS
    c = CONFIGS["tto10k"]
    sg = _grid("tto10k", c["n_tight"])
    g = Grid(sg)
    topo = random_topologies(sg, c["batch"], seed=1)
    t = torch.tensor(topo, dtype=torch.int32, device="cuda")
    wk = g.worst_k(t, k=20, all_energy=True)
    bb = g.busbar(t, bmax=True)
    g.sync_status()
    i = next(j for j in range(64) if dcflow.is_connected_uf(*dcflow.post_split_graph(sg, topo[j])[:3]))
    r = dcflow.evaluate_parallel_outages(sg, topo[i], processes=parity.n_procs(), want_energy=True)
    out = {"all_energy": wk["all_energy"][i:i + 1].cpu().numpy(), "outage": wk["outage"][i:i + 1].cpu().numpy(),
           "energy": wk["energy"][i:i + 1].cpu().numpy()}
    _check(sg, out, [0], [r["outage_energy"]], 20)
    rb = dcflow.busbar_outages(sg, topo[i])
    lim = sg.limit[sg.monitored.astype(np.int64)]
    bm = bb["bmax"][i].cpu().numpy().astype(np.float64)
    err = np.abs(bm - rb["bmax"]) / lim[None, :]
    allowed = parity.TOL_FP32 + parity.FLOW_ULPS * np.abs(rb["bmax"]) / lim[None, :]
    assert np.all(err <= allowed), float(err.max())
    assert int(bb["n_island"][i]) == rb["n_islanded_busbar"]
