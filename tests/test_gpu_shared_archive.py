"""The shared-repertoire step (paper_2605_10128_b300.shared_archive) on one
GPU: two archive replicas stand for two ranks.  Each proposes with its rank's
key from its own copy, the library evaluates the proposals, the rows are
concatenated in rank order (what the all-gather returns) and inserted into
both replicas.  The replicas must stay bit-identical, every batch of proposals
must equal the oracle's from the same archive, and the archive must equal the
oracle's sequential insert of the gathered batch (Algorithm 3).  With one
rank the shared step equals the library's fused MapElites step."""
import numpy as np
import pytest

from oracle import dcflow, mapelites as me
from synth import config_grid, limits_from_flows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED, B, ITERS = 41, 96, 8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _grid():
    sg = config_grid("tto30")
    return sg.with_limits(limits_from_flows(dcflow.base_flows(sg)[0], 5))


def _same_archive(oracle_arch, export):
    fit, gen, filled = export
    assert set(np.flatnonzero(filled)) == set(oracle_arch.elites)
    for c, (f, g) in oracle_arch.elites.items():
        assert fit[c] == np.float32(f)
        np.testing.assert_array_equal(gen[c], g)


def test_two_replicas_stay_identical():
    from paper_2605_10128_b300 import Grid, Archive
    from paper_2605_10128_b300.shared_archive import pack_rows, unpack_rows, rank_key
    sg = _grid()
    g = Grid(sg)
    reps = [Archive(g, 8, 8), Archive(g, 8, 8)]
    ref = me.Archive(8, 8)
    tab = me.ActionTable(sg)
    for it in range(ITERS):
        rows = []
        for r, a in enumerate(reps):
            topo = a.propose(rank_key(SEED, r), it, B)
            np.testing.assert_array_equal(topo.cpu().numpy(), me.propose(ref, tab, rank_key(SEED, r), it, B,
                                                                           sg.k_max))
            out = g.evaluate(topo)
            rows.append(pack_rows(topo, out["fitness"], out["cell"]))
        gathered = torch.cat(rows)
        for a in reps:
            a.insert(*unpack_rows(gathered))
        g.sync_status()
        e0, e1 = reps[0].export(), reps[1].export()
        for x, y in zip(e0, e1):
            assert np.array_equal(x, y)
        t, f, c = unpack_rows(gathered.cpu())
        ref.insert(c.numpy(), f.numpy().astype(np.float64), t.numpy())
        _same_archive(ref, e0)
    assert len(ref.elites) > 3


def test_single_rank_shared_step_equals_fused_step():
    from paper_2605_10128_b300 import Grid, Archive
    from paper_2605_10128_b300.shared_archive import SharedArchive
    sg = _grid()
    g = Grid(sg)
    a, b = Archive(g, 8, 8), Archive(g, 8, 8)
    sa = SharedArchive(b)
    for it in range(ITERS):
        a.step(SEED, it, B)
        rows = sa.step(SEED, it, B)
        assert tuple(rows.shape) == (B, sg.k_max + 2)
    g.sync_status()
    for x, y in zip(a.export(), b.export()):
        assert np.array_equal(x, y)
