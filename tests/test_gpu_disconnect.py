"""Branch-disconnection slots (Sec. "Repertoire design"), the lambda_d cell
and crossover (Algorithm 2) on the GPU against the oracle: evaluation parity in
FP32 and on the tcgen05 TF32 sweep, the edge cases of opened branches, bit-exact
proposals with and without crossover, and a MapElites run over the
three-dimensional archive."""
import numpy as np
import pytest

from oracle import dcflow
from oracle import mapelites as me
from synth import config_grid, limits_from_flows, random_topologies
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MUT = (0.2, 0.2, 0.5, 0.1, 2.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _grid(name, n_disc, n_dslot, n_tight, seed=0):
    sg = config_grid(name, seed=seed, n_disc=n_disc, n_dslot=n_dslot)
    f0 = dcflow.base_flows(sg)
    return sg.with_limits(limits_from_flows(f0[0], n_tight, seed=seed))


def _run(g, topo, prec, d_disc, shape=-1):
    g.set_sweep_shape(prec, shape)
    out = g.evaluate(torch.tensor(topo, dtype=torch.int32, device="cuda"), precision=prec, metrics=True,
                     fmax=True, d_disc=d_disc)
    g.sync_status()
    g.set_sweep_shape(prec, -1)
    return {k: v.cpu().numpy() for k, v in out.items() if not k.startswith("_")}


def _special_rows(sg):
    """Genomes for the edge cases: only disconnections; a split that moves an
    opened branch (with another branch left on busbar B, and with none); and
    the unchanged topology."""
    k = sg.k_max
    rows = []
    row = np.full(sg.genome_width, -1, dtype=np.int32)
    row[k] = 0
    row[k + 1] = 1
    rows.append(row)
    disc = {int(e): j for j, e in enumerate(sg.disc)}
    kinds = set()
    for a in range(sg.n_action):
        s = int(sg.action_station[a])
        assets = sg.station_assets(s)
        mask = int(sg.action_mask[a])
        on_b = [int(assets[i]) for i in range(len(assets)) if (mask >> i) & 1 and assets[i] >= 0]
        hit = [e for e in on_b if e in disc]
        if not hit:
            continue
        kind = len(on_b) == 1
        if kind in kinds:
            continue
        kinds.add(kind)
        row = np.full(sg.genome_width, -1, dtype=np.int32)
        row[0] = a
        row[k] = disc[hit[0]]
        rows.append(row)
    rows.append(np.full(sg.genome_width, -1, dtype=np.int32))
    return np.stack(rows), kinds


@pytest.mark.parametrize("prec,shape", [(0, -1), (3, 4), (3, 0)])
def test_disconnections_match_oracle_30bus(prec, shape):
    from paper_2605_10128_b300 import Grid
    sg = _grid("tto30", 12, 2, 5)
    g = Grid(sg)
    assert g.genome_width == sg.k_max + 2 and g.n_disc == 12
    special, kinds = _special_rows(sg)
    assert kinds == {True, False}
    topo = np.concatenate([special, random_topologies(sg, 120, seed=3)])
    idx = list(range(len(topo)))
    refs = parity.oracle_eval(sg, topo, idx, d_disc=3)
    out = _run(g, topo, prec, 3, shape)
    parity.compare(sg, out, idx, refs)
    # the split whose busbar B keeps only an opened branch islands the grid
    assert any(r["island_base"] for r in refs[: len(special)])
    assert sum(r["nd"] > 0 for r in refs) > 60


def test_disconnections_tto2k_sampled():
    from paper_2605_10128_b300 import Grid
    sg = _grid("tto2k", 60, 2, 30)
    g = Grid(sg)
    topo = random_topologies(sg, 512, seed=8)
    idx = [0, 1, 2, 3, 5, 8]
    refs = parity.oracle_eval(sg, topo, idx, d_disc=3)
    assert any(r["nd"] > 0 for r in refs)
    for prec, shape in [(0, -1), (3, 4)]:
        out = _run(g, topo, prec, 3, shape)
        parity.compare(sg, out, idx, refs)


def test_invalid_disconnections_reported():
    from paper_2605_10128_b300 import Grid, TTOError
    sg = _grid("tto30", 6, 2, 5)
    g = Grid(sg)
    k = sg.k_max
    for bad in ([-1] * k + [2, 2], [-1] * k + [6, -1]):
        out = g.evaluate(torch.tensor([bad], dtype=torch.int32, device="cuda"))
        with pytest.raises(TTOError) as ei:
            g.sync_status()
        assert ei.value.code == -5
        assert out["fitness"][0].item() == -np.inf
    g.sync_status()


def _random_archive(sg, ds, dm, dd, n_fill, seed):
    rng = np.random.default_rng(seed)
    cells = ds * dm * dd
    gens = random_topologies(sg, n_fill, seed=seed, min_splits=0)
    fit = np.full(cells, -np.inf, dtype=np.float32)
    gen = np.full((cells, sg.genome_width), -1, dtype=np.int32)
    filled = np.zeros(cells, dtype=np.uint8)
    arch = me.Archive(ds, dm, dd)
    for gg in gens:
        _, _, c = dcflow.descriptors(sg, gg, ds, dm, dd)
        f = np.float32(-rng.random() * 100)
        fit[c], gen[c], filled[c] = f, gg, 1
        arch.elites[c] = (float(f), gg.copy())
    return fit, gen, filled, arch


@pytest.mark.parametrize("cross,p_c1", [(0, 0.5), (1, 0.5), (1, 1.0), (1, 0.0), (1, 0.3)])
def test_proposals_with_disconnections_bit_exact(cross, p_c1):
    from paper_2605_10128_b300 import Grid, Archive
    sg = _grid("tto2k", 60, 3, 30)
    g = Grid(sg)
    A = Archive(g, 8, 8, 3)
    fit, gen, filled, arch = _random_archive(sg, 8, 8, 3, 60, seed=4)
    A.load(fit, gen, filled)
    tab = me.ActionTable(sg)
    dprobs = (0.25, 0.25, 0.5, 0.0)
    mut = MUT + dprobs + (cross, p_c1)
    for it in [0, 7, 2 ** 33 + 1]:
        got = A.propose(99, it, 700, mutation=mut).cpu().numpy()
        ref = me.propose(arch, tab, 99, it, 700, sg.k_max, probs=MUT[:4], mean=MUT[4], n_dslot=3,
                         n_disc=sg.n_disc, dprobs=dprobs, crossover_on=bool(cross), p_c1=p_c1)
        np.testing.assert_array_equal(got, ref)
    if cross:
        assert me.mutation_count(99, 7, 700, True) < 700 or me.mutation_count(99, 0, 700, True) < 700


def test_mapelites_run_with_disconnections_and_crossover():
    """Fused iterations on the 30-bus grid with two disconnection slots, a
    3-valued lambda_d axis and crossover: every proposal batch equals the
    oracle's from the GPU archive it starts from, and every filled cell's
    elite has that cell's descriptors."""
    from paper_2605_10128_b300 import Grid, Archive
    sg = _grid("tto30", 12, 2, 5)
    g = Grid(sg)
    ds, dm, dd = 8, 8, 3
    A = Archive(g, ds, dm, dd)
    tab = me.ActionTable(sg)
    B = 256
    mut = MUT + (0.25, 0.25, 0.5, 0.0, 1, 0.5)
    topo_t = torch.empty(B, sg.genome_width, dtype=torch.int32, device="cuda")
    fit_t = torch.empty(B, dtype=torch.float32, device="cuda")
    for it in range(12):
        f, gen, fl = A.export()
        arch = me.Archive(ds, dm, dd)
        for c in np.flatnonzero(fl):
            arch.elites[int(c)] = (float(f[c]), gen[c].copy())
        ref = me.propose(arch, tab, 5, it, B, sg.k_max, probs=MUT[:4], mean=MUT[4], n_dslot=2,
                         n_disc=sg.n_disc, crossover_on=True, p_c1=0.5)
        A.step(5, it, B, mutation=mut, topo_out=topo_t, fitness_out=fit_t)
        g.sync_status()
        np.testing.assert_array_equal(topo_t.cpu().numpy(), ref)
    f, gen, fl = A.export()
    assert fl.sum() > 20
    assert any(dcflow.descriptors(sg, gen[c], ds, dm, dd)[2] % dd > 0 for c in np.flatnonzero(fl))
    for c in np.flatnonzero(fl):
        assert dcflow.descriptors(sg, gen[c], ds, dm, dd)[2] == c
