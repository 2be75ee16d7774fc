"""GPU parity of tto_evaluate_batch against the FP64 brute-force oracle."""
import numpy as np
import pytest

from oracle import dcflow
from synth import config_grid, limits_from_flows, make_grid, random_topologies, CONFIGS
from tests.gridcases import three_bus, action_of
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def lib_grid(sg):
    from paper_2605_10128_b300 import Grid
    return Grid(sg)


def run(g, topo, **kw):
    t = torch.as_tensor(np.ascontiguousarray(topo), dtype=torch.int32).cuda()
    out = g.evaluate(t, metrics=True, fmax=True, **kw)
    g.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items() if not k.startswith("_")}


def with_limits(sg, n_tight):
    f0 = dcflow.base_flows(sg)
    return sg.with_limits(limits_from_flows(f0[0], n_tight, seed=sg.seed))


def test_three_bus_golden_through_library():
    sg, d = three_bus()
    g = lib_grid(sg)
    a2, a6 = action_of(sg, 0, 2), action_of(sg, 0, 6)
    out = run(g, np.array([[-1], [a2], [a6]], dtype=np.int32))
    base = d["cases"]["base"]
    np.testing.assert_allclose(out["fmax"][0, 0], base["fmax"], atol=1e-6)
    assert out["fitness"][0] == pytest.approx(base["fitness"], abs=1e-5)
    np.testing.assert_allclose(out["metrics"][0], [base["lambda_o"], base["maxload"],
                                                   base["lambda_c"], base["lambda_c0"]], atol=1e-5)
    assert list(out["island"]) == [0, 2, 2]
    np.testing.assert_array_equal(out["fmax"][1:], 0.0)
    # N-0 loadings of the two split states: max(|f'|/limit)
    lim = np.array(sg.limit)
    for i, case in [(1, "split_branch_only"), (2, "split_branch_and_injection")]:
        fp = np.abs(np.array(d["cases"][case]["fprime"]))
        assert out["metrics"][i][1] == pytest.approx(float((fp / lim).max()), abs=1e-6)
    assert list(out["cell"]) == [0, 9, 9]


# FP32 flows with an FP32 or TF32-split low-rank term meet the FP32 bar; the
# 16-bit splits meet the BF16 bar (their measured error is printed).
# The tcgen05 sweep (TF32X3 sweep variant 4) is held to the same FP32 bar.
# FP16X3 (an experimental split, not a mode of the workload) and the plain BF16
# product are held to the structural checks and their loading error reported:
# fp16's 5-bit exponent loses small entries of U and V, and FP16X3 missed the
# BF16 bar on 1 of 64 sampled 2000-bus topologies (8e-3 of the limit).
PRECISIONS = [("fp32", 0, parity.TOL_FP32, None), ("tf32x3", 3, parity.TOL_FP32, None),
              ("tf32x3 tcgen05", 3, parity.TOL_FP32, 4), ("fp16x3", 4, np.inf, None),
              ("bf16x3", 1, parity.TOL_BF16, None)]


def check_all_precisions(label, sg, g, topo, idx, refs, plain_bf16=True, **kw):
    """Every precision mode against the same oracle results; the report-only
    modes are held to the structural checks and their loading error reported."""
    for name, prec, tol, shape in PRECISIONS:
        if shape is not None:
            g.set_sweep_shape(prec, shape)
        try:
            out = run(g, topo, precision=prec, **kw)
        finally:
            if shape is not None:
                g.set_sweep_shape(prec, -1)
        split = {}
        worst = parity.compare(sg, out, idx, refs, tol=tol, split=split)
        print(f"{label} {name} worst loading error {worst:.2e} of limit; "
              + parity.split_report(split, tol if np.isfinite(tol) else parity.TOL_BF16))
    if plain_bf16:
        out = run(g, topo, precision=2, **kw)
        worst = parity.compare(sg, out, idx, refs, tol=np.inf)
        print(f"{label} bf16 (single product) worst loading error {worst:.2e} of limit")


def test_tto30_every_topology():
    sg = with_limits(config_grid("tto30"), CONFIGS["tto30"]["n_tight"])
    topo = random_topologies(sg, 256, seed=11)
    topo[0] = -1  # the unsplit topology
    g = lib_grid(sg)
    idx = list(range(256))
    refs = parity.oracle_eval(sg, topo, idx)
    check_all_precisions("tto30", sg, g, topo, idx, refs)
    assert sum(r["island_base"] for r in refs) > 0  # the batch exercises split islanding
    assert sum(r["island_any"] for r in refs) > 0


@pytest.mark.parametrize("seed", [3, 4])
def test_ragged_tiles_subsets_and_timesteps(seed):
    """Several row tiles with a ragged tail, outage and monitored subsets, a
    ragged batch, and a reordered timestep subset."""
    sg = make_grid(300, 450, 24, assets=(4, 8), T=3, b_dist=("loguniform", 2.0, 200.0),
                   noise=0.1, seed=seed, k_max=3, name="rag")
    rng = np.random.default_rng(seed)
    sg.monitored = np.sort(rng.choice(450, 333, replace=False)).astype(np.int32)
    sg.outages = np.sort(rng.choice(450, 201, replace=False)).astype(np.int32)
    sg = with_limits(sg, 5)
    topo = random_topologies(sg, 37, seed=seed)
    g = lib_grid(sg)
    for ts in [None, [2, 0]]:
        idx = list(range(37))
        refs = parity.oracle_eval(sg, topo, idx, timesteps=ts)
        check_all_precisions(f"ragged{seed} t={ts}", sg, g, topo, idx, refs, timesteps=ts)


@pytest.mark.parametrize("T", [24, 9])
def test_long_horizons(T):
    """Timestep counts that the tensor-core sweep splits into passes (24 = 3 x 8)
    or pads (9 -> 16)."""
    sg = make_grid(120, 180, 10, assets=(4, 8), T=T, b_dist=("loguniform", 2.0, 200.0),
                   noise=0.1, seed=T, k_max=4, name="long")
    sg = with_limits(sg, 3)
    topo = random_topologies(sg, 20, seed=T)
    g = lib_grid(sg)
    idx = list(range(20))
    refs = parity.oracle_eval(sg, topo, idx)
    check_all_precisions(f"T={T}", sg, g, topo, idx, refs)


def test_fitness_f1_option():
    sg = with_limits(config_grid("tto30", seed=2), 5)
    topo = random_topologies(sg, 64, seed=5)
    g = lib_grid(sg)
    from paper_2605_10128_b300 import FIT_F1
    out = run(g, topo, fitness_kind=FIT_F1)
    idx = list(range(64))
    refs = parity.oracle_eval(sg, topo, idx)
    parity.compare(sg, out, idx, refs, fitness_kind=1)


def test_tto2k_sampled_against_oracle():
    sg = with_limits(config_grid("tto2k"), CONFIGS["tto2k"]["n_tight"])
    topo = random_topologies(sg, 512, seed=21)
    g = lib_grid(sg)
    idx = [0, 1, 2, 3]
    refs = parity.oracle_eval(sg, topo, idx)
    check_all_precisions("tto2k", sg, g, topo, idx, refs)


@pytest.mark.slow
def test_tto2k_64_sampled_topologies_against_oracle():
    """The 2000-bus precision workload: 64 topologies of a 4096 batch against
    the oracle over all 3000 outages and 16 timesteps, every precision mode
    (worst error per mode printed)."""
    sg = with_limits(config_grid("tto2k"), CONFIGS["tto2k"]["n_tight"])
    topo = random_topologies(sg, CONFIGS["tto2k"]["batch"], seed=22)
    g = lib_grid(sg)
    idx = list(range(0, CONFIGS["tto2k"]["batch"], 64))
    refs = parity.oracle_eval(sg, topo, idx)
    check_all_precisions("tto2k x64", sg, g, topo, idx, refs)


@pytest.mark.slow
def test_tto10k_full_batch_sampled_against_oracle():
    """The 10000-bus workload in the benchmark's launch configuration (8192
    topologies, 5000 outages x 15000 monitored, 4 timesteps); one non-islanded
    and one islanded topology re-solved by the oracle over every outage."""
    c = CONFIGS["tto10k"]
    sg = with_limits(config_grid("tto10k"), c["n_tight"])
    topo = random_topologies(sg, c["batch"], seed=1)
    g = lib_grid(sg)
    picks = []
    want_isl = True
    for i in range(64):
        n_node, fr, to, _, _ = dcflow.post_split_graph(sg, topo[i])
        conn = dcflow.is_connected_uf(n_node, fr, to)
        if conn and len([p for p in picks if p[1]]) < 1:
            picks.append((i, True))
        elif not conn and want_isl:
            picks.append((i, False))
            want_isl = False
        if len(picks) == 2:
            break
    idx = [p[0] for p in picks]
    refs = [dcflow.evaluate_parallel_outages(sg, topo[i], processes=parity.n_procs(), d_split=20,
                                             d_moved=20) for i in idx]
    check_all_precisions("tto10k", sg, g, topo, idx, refs, d_split=20, d_moved=20)
    out = run(g, topo, d_split=20, d_moved=20, precision=1)
    # every cell of the batch matches the oracle's descriptor mapping
    for i in range(0, c["batch"], 97):
        ns, nm, cell = dcflow.descriptors(sg, topo[i], 20, 20)
        assert int(out["cell"][i]) == cell and tuple(out["desc"][i]) == (ns, nm)


def test_invalid_genomes_reported():
    sg = with_limits(config_grid("tto30"), 5)
    g = lib_grid(sg)
    a0 = int(sg.action_offset[0])
    from paper_2605_10128_b300 import TTOError
    for bad in ([a0, a0 + 1], [sg.n_action, -1]):
        t = torch.tensor([bad], dtype=torch.int32, device="cuda")
        out = g.evaluate(t)
        with pytest.raises(TTOError) as ei:
            g.sync_status()
        assert ei.value.code == -5
        assert out["fitness"][0].item() == -np.inf
    g.sync_status()  # cleared


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_deterministic_and_order_independent(prec):
    sg = with_limits(config_grid("tto30", seed=4), 5)
    topo = random_topologies(sg, 200, seed=8)
    g = lib_grid(sg)
    a = run(g, topo, precision=prec)
    b = run(g, topo, precision=prec)
    perm = np.random.default_rng(0).permutation(200)
    c = run(g, topo[perm], precision=prec)
    for k in ["fitness", "desc", "cell", "island", "metrics", "fmax"]:
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k][perm], c[k])


def test_empty_batch_and_validation():
    sg = with_limits(config_grid("tto30"), 5)
    g = lib_grid(sg)
    from paper_2605_10128_b300 import TTOError
    t = torch.zeros(0, sg.k_max, dtype=torch.int32, device="cuda")
    g.evaluate(t)
    g.sync_status()
    with pytest.raises(TTOError):
        g.evaluate(torch.zeros(4, sg.k_max, dtype=torch.int32, device="cuda"), timesteps=[5])


@pytest.mark.slow
def test_tto10k_full_rows_sampled_outages_many_topologies():
    """The 10000-bus grid with all 15000 monitored branches and 4 timesteps
    but 120 sampled non-bridge outages, so that the oracle can re-solve many
    topologies: 40 topologies of an 8192 batch (every split count 1 to 6, and
    4 that island the grid) in FP32, the tcgen05 TF32X3 sweep, every mma.sync
    variant and the BF16 split, with the error split into near-limit and
    far-above-limit parts."""
    from dataclasses import replace
    c = CONFIGS["tto10k"]
    full = with_limits(config_grid("tto10k"), c["n_tight"])
    rng = np.random.default_rng(12)
    sg = replace(full, outages=np.sort(rng.choice(full.outages, 120, replace=False)).astype(np.int32))
    topo = random_topologies(sg, c["batch"], seed=3)
    per_k = {k: [] for k in range(1, 7)}
    isl = []
    for i in range(c["batch"]):
        n_node, fr, to, _, _ = dcflow.post_split_graph(sg, topo[i])
        if not dcflow.is_connected_uf(n_node, fr, to):
            if len(isl) < 4:
                isl.append(i)
            continue
        k = int((topo[i] >= 0).sum())
        if len(per_k[k]) < 6:
            per_k[k].append(i)
        if len(isl) == 4 and all(len(v) == 6 for v in per_k.values()):
            break
    idx = sorted(isl + [i for v in per_k.values() for i in v])
    assert len(isl) == 4 and len(idx) == 40
    refs = parity.oracle_eval(sg, topo, idx, d_split=20, d_moved=20)
    g = lib_grid(sg)
    check_all_precisions("tto10k rows x 120 outages", sg, g, topo, idx, refs, plain_bf16=False,
                         d_split=20, d_moved=20)
    for variant in range(4):  # every mma.sync tile variant of TF32X3
        g.set_sweep_shape(3, variant)
        out = run(g, topo, precision=3, d_split=20, d_moved=20)
        split = {}
        worst = parity.compare(sg, out, idx, refs, tol=parity.TOL_FP32, split=split)
        print(f"tto10k rows x 120 outages tf32x3 mma.sync variant {variant}: worst {worst:.2e}; "
              + parity.split_report(split, parity.TOL_FP32))
    g.set_sweep_shape(3, -1)
