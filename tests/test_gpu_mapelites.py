"""GPU MapElites operators against the oracle: Philox words, proposals
(bit-exact genomes), scatter insert vs the sequential insert, and a 20-iteration
trajectory on the 30-bus workload compared up to the first near-tie."""
import numpy as np
import pytest

from oracle import dcflow
from oracle import mapelites as me
from oracle.philox import philox4x32_10
from synth import config_grid, limits_from_flows, random_topologies, CONFIGS
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def grid30(seed=0):
    sg = config_grid("tto30", seed=seed)
    f0 = dcflow.base_flows(sg)
    return sg.with_limits(limits_from_flows(f0[0], 5, seed=seed))


def test_philox_blocks_bit_exact():
    from paper_2605_10128_b300 import philox_blocks
    for seed, it, cand in [(0, 0, 0), (0xDEADBEEFCAFE, 123456789012, 77), (2 ** 64 - 1, 2 ** 40, 2 ** 31)]:
        out = philox_blocks(seed, it, cand, 5, 20).cpu().numpy().view(np.uint32)
        for i in range(20):
            ref = philox4x32_10((5 + i, cand, it & 0xFFFFFFFF, it >> 32), (seed & 0xFFFFFFFF, seed >> 32))
            assert tuple(int(x) for x in out[i]) == ref


def _random_archive(sg, d_split, d_moved, n_fill, seed):
    rng = np.random.default_rng(seed)
    cells = d_split * d_moved
    gens = random_topologies(sg, n_fill, seed=seed, min_splits=0)
    fit = np.full(cells, -np.inf, dtype=np.float32)
    gen = np.full((cells, sg.k_max), -1, dtype=np.int32)
    filled = np.zeros(cells, dtype=np.uint8)
    arch = me.Archive(d_split, d_moved)
    for gg in gens:
        _, _, c = dcflow.descriptors(sg, gg, d_split, d_moved)
        f = np.float32(-rng.random() * 100)
        fit[c], gen[c], filled[c] = f, gg, 1
        arch.elites[c] = (float(f), gg.copy())
    return fit, gen, filled, arch


@pytest.mark.parametrize("mut", [(0.2, 0.2, 0.5, 0.1, 2.0), (0.6, 0.1, 0.2, 0.1, 3.0),
                                 (0.3, 0.3, 0.4, 0.0, 1.0)])
def test_proposals_bit_exact(mut):
    from paper_2605_10128_b300 import Grid, Archive
    sg = config_grid("tto2k")
    sg = sg.with_limits(np.ones(sg.n_branch))
    g = Grid(sg)
    A = Archive(g, 8, 8)
    fit, gen, filled, arch = _random_archive(sg, 8, 8, 40, seed=3)
    A.load(fit, gen, filled)
    tab = me.ActionTable(sg)
    for it in [0, 1, 2 ** 33 + 5]:
        got = A.propose(1234, it, 300, mutation=mut).cpu().numpy()
        ref = me.propose(arch, tab, 1234, it, 300, sg.k_max, probs=mut[:4], mean=mut[4])
        np.testing.assert_array_equal(got, ref)


def test_proposals_from_empty_archive():
    from paper_2605_10128_b300 import Grid, Archive
    sg = grid30()
    g = Grid(sg)
    A = Archive(g, 8, 8)
    got = A.propose(9, 0, 256).cpu().numpy()
    ref = me.propose(me.Archive(8, 8), me.ActionTable(sg), 9, 0, 256, sg.k_max)
    np.testing.assert_array_equal(got, ref)
    assert np.all((got >= 0).sum(axis=1) >= 1)


def test_scatter_insert_equals_sequential():
    from paper_2605_10128_b300 import Grid, Archive
    sg = grid30()
    g = Grid(sg)
    rng = np.random.default_rng(5)
    for trial in range(5):
        A = Archive(g, 4, 4)
        fit0, gen0, filled0, arch = _random_archive(sg, 4, 4, 6, seed=trial)
        A.load(fit0, gen0, filled0)
        B = 500
        topo = random_topologies(sg, B, seed=trial + 100)
        cells = rng.integers(0, 16, B).astype(np.int32)
        fit = -rng.integers(0, 40, B).astype(np.float32)  # many exact ties
        fit[rng.random(B) < 0.05] = -np.inf
        fit[:3] = fit0[cells[:3]]  # ties with incumbents
        A.insert(torch.tensor(topo).cuda(), torch.tensor(fit).cuda(), torch.tensor(cells).cuda())
        arch.insert(cells, fit, topo)
        f, gg, fl = A.export()
        for c in range(16):
            if c in arch.elites:
                assert fl[c] == 1 and f[c] == np.float32(arch.elites[c][0])
                np.testing.assert_array_equal(gg[c], arch.elites[c][1])
            else:
                assert fl[c] == 0


def test_mapelites_trajectory_tto30():
    """20 fused iterations (propose, exact evaluation, insert) against the
    oracle, compared while no insert decision is a near-tie."""
    from paper_2605_10128_b300 import Grid, Archive
    c = CONFIGS["tto30"]
    sg = grid30()
    g = Grid(sg)
    ds, dm = c["archive"]
    A = Archive(g, ds, dm)
    arch = me.Archive(ds, dm)
    tab = me.ActionTable(sg)
    B = c["batch"]
    lim_sum = float(sg.limit.sum())
    tol = parity.TOL_FP32 * lim_sum + parity.TOL_FP32
    topo_t = torch.empty(B, sg.k_max, dtype=torch.int32, device="cuda")
    fit_t = torch.empty(B, dtype=torch.float32, device="cuda")
    compared = 0
    for it in range(c["iterations"]):
        ref_topo = me.propose(arch, tab, 77, it, B, sg.k_max)
        A.step(77, it, B, topo_out=topo_t, fitness_out=fit_t)
        g.sync_status()
        got_topo = topo_t.cpu().numpy()
        np.testing.assert_array_equal(got_topo, ref_topo)
        res = dcflow.evaluate_many(sg, list(ref_topo), processes=parity.n_procs(), d_split=ds, d_moved=dm)
        fref = np.array([r["fitness"] for r in res])
        fgot = fit_t.cpu().numpy().astype(np.float64)
        fin = np.isfinite(fref)
        assert np.array_equal(fin, np.isfinite(fgot))
        err = float(np.max(np.abs(fgot[fin] - fref[fin]), initial=0.0))
        assert err <= tol
        # every FP32 fitness is within err of its FP64 value, so an FP64 gap
        # wider than 2 err between different genomes fixes the GPU's decision
        # too; a narrower gap is a near-tie that ends the comparison
        gap = 2.0 * err + 1e-12
        cells = np.array([r["cell"] for r in res])
        tie = False
        for cc in np.unique(cells[fin]):
            ids = np.flatnonzero(fin & (cells == cc))
            top = ids[np.argmax(fref[ids])]
            for j in ids:
                if j == top or np.array_equal(ref_topo[j], ref_topo[top]):
                    continue
                if fref[j] == fref[top] and fgot[j] == fgot[top]:
                    continue  # exact tie on both sides: both keep the lower index
                if fref[top] - fref[j] <= gap:
                    tie = True
            inc = arch.elites.get(int(cc))
            if inc is not None and abs(fref[top] - inc[0]) <= gap and not np.array_equal(inc[1], ref_topo[top]):
                tie = True
        arch.insert(cells, fref, ref_topo)
        if tie:
            break
        f, gg, fl = A.export()
        assert set(np.flatnonzero(fl)) == set(arch.elites)
        for cc, (fv, gv) in arch.elites.items():
            np.testing.assert_array_equal(gg[cc], gv)
            assert abs(float(f[cc]) - fv) <= tol
        # continue from identical archives: the oracle takes the GPU's fitness
        arch.elites = {int(cc): (float(f[cc]), gg[cc].copy()) for cc in np.flatnonzero(fl)}
        compared += 1
    print(f"tto30 MapElites iterations compared: {compared}")
    assert compared >= 3
