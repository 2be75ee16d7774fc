"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
hand-derived closed forms (3-bus golden file), Kirchhoff's current and voltage
laws, bridges found by an independent library (networkx), an independent FP64
restatement of the PTDF/LODF/bus-split low-rank formulas, and the projection
invariants of the flow-response matrix."""
import numpy as np
import networkx as nx
import pytest

from oracle import dcflow
from synth import limits_from_flows, random_topologies
from tests.gridcases import three_bus, small_grid, action_of


def test_three_bus_closed_form():
    g, d = three_bus()
    base = d["cases"]["base"]
    r = dcflow.evaluate(g, [-1], want_flows=True)
    np.testing.assert_allclose(r["fprime"][0], base["fprime"], atol=1e-14)
    for c, fl in base["outage_flows"].items():
        np.testing.assert_allclose(r["per_outage"][int(c)][0], fl, atol=1e-14)
    np.testing.assert_allclose(r["fmax"][0], base["fmax"], atol=1e-14)
    assert r["n_islanded"] == base["n_islanded"]
    assert r["lambda_o"] == pytest.approx(base["lambda_o"], abs=1e-14)
    assert r["lambda_c"] == base["lambda_c"]
    assert r["lambda_c0"] == base["lambda_c0"]
    assert r["maxload"] == pytest.approx(base["maxload"], abs=1e-14)
    assert r["fitness"] == pytest.approx(base["fitness"], abs=1e-14)
    assert r["lambda_f1"] == pytest.approx(base["lambda_f1"], abs=1e-14)


@pytest.mark.parametrize("case", ["split_branch_only", "split_branch_and_injection"])
def test_three_bus_splits(case):
    g, d = three_bus()
    c = d["cases"][case]
    a = action_of(g, 0, c["mask"])
    r = dcflow.evaluate(g, [a])
    assert not r["island_base"]
    np.testing.assert_allclose(r["fprime"][0], c["fprime"], atol=1e-14)
    assert r["n_islanded"] == c["n_islanded"]
    assert r["island_any"]
    # every outage islands: nothing enters the N-1 maximum
    np.testing.assert_array_equal(r["fmax"], 0.0)


def _kcl_kvl(n_node, fr, to, b, p, slack, flows, skip=-1, opened=()):
    E = len(fr)
    out = set(opened) | {skip}
    net = np.zeros((p.shape[0], n_node))
    for l in range(E):
        if l in out:
            continue
        net[:, fr[l]] += flows[:, l]
        net[:, to[l]] -= flows[:, l]
    others = [i for i in range(n_node) if i != slack]
    np.testing.assert_allclose(net[:, others], p[:, others], atol=1e-9)
    np.testing.assert_allclose(net.sum(axis=1), 0.0, atol=1e-9)
    G = nx.Graph()
    G.add_nodes_from(range(n_node))
    for l in range(E):
        if l not in out:
            G.add_edge(int(fr[l]), int(to[l]), l=l)
    for cyc in nx.cycle_basis(G):
        s = np.zeros(p.shape[0])
        for i in range(len(cyc)):
            u, v = cyc[i], cyc[(i + 1) % len(cyc)]
            l = G[u][v]["l"]
            sign = 1.0 if (fr[l] == u and to[l] == v) else -1.0
            s += sign * flows[:, l] / b[l]
        np.testing.assert_allclose(s, 0.0, atol=1e-9)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kirchhoff_laws_every_state(seed):
    """KCL at every node (split busbars included) and KVL around every cycle,
    in the N-0 state and in every non-islanding outage state."""
    g = small_grid(seed)
    topo = random_topologies(g, 4, seed=seed)
    for gen in topo:
        n_node, fr, to, p, _ = dcflow.post_split_graph(g, gen)
        if not dcflow.is_connected_uf(n_node, fr, to):
            continue
        f = dcflow.solve_flows(n_node, fr, to, g.b, p, g.slack)
        _kcl_kvl(n_node, fr, to, g.b, p, g.slack, f)
        for c in range(len(fr)):
            if not dcflow.is_connected_uf(n_node, fr, to, skip=c):
                continue
            F = dcflow.solve_flows(n_node, fr, to, g.b, p, g.slack, skip=c)
            assert np.all(F[:, c] == 0.0)
            _kcl_kvl(n_node, fr, to, g.b, p, g.slack, F, skip=c)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_islanding_matches_networkx_bridges(seed):
    g = small_grid(seed)
    g = g.with_limits(np.ones(g.n_branch))
    topo = random_topologies(g, 6, seed=seed)
    for gen in topo:
        n_node, fr, to, p, _ = dcflow.post_split_graph(g, gen)
        G = nx.Graph()
        G.add_nodes_from(range(n_node))
        for l in range(len(fr)):
            G.add_edge(int(fr[l]), int(to[l]), l=l)
        r = dcflow.evaluate(g, gen)
        assert r["island_base"] == (not nx.is_connected(G))
        if r["island_base"]:
            continue
        bridges = {G[u][v]["l"] for u, v in nx.bridges(G)}
        n_br = sum(1 for c in g.outages if int(c) in bridges)
        assert r["n_islanded"] == n_br


def _ptdf_restatement(g):
    """Independent dense FP64 statement of PTDF = D A X and N = I - D A X A^T."""
    n, E = g.n_bus, g.n_branch
    A = np.zeros((E, n))
    A[np.arange(E), g.from_bus] = 1.0
    A[np.arange(E), g.to_bus] = -1.0
    D = np.diag(g.b)
    idx = [i for i in range(n) if i != g.slack]
    Br = (A.T @ D @ A)[np.ix_(idx, idx)]
    X = np.zeros((n, n))
    X[np.ix_(idx, idx)] = np.linalg.inv(Br)
    M = D @ A @ X @ A.T
    return A, D, X, M


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_flow_response_invariants(seed):
    g = small_grid(seed)
    A, D, X, M = _ptdf_restatement(g)
    N = np.eye(g.n_branch) - M
    np.testing.assert_allclose(M @ M, M, atol=1e-10)
    assert np.trace(M) == pytest.approx(g.n_bus - 1, abs=1e-9)
    ND = N @ D
    np.testing.assert_allclose(ND, ND.T, atol=1e-9)
    assert np.linalg.eigvalsh((ND + ND.T) / 2).min() > -1e-9
    d = np.diag(N)
    assert d.min() > -1e-12 and d.max() < 1 + 1e-12
    # the oracle's own solve reproduces the M columns: unit transfer across c
    for c in range(g.n_branch):
        p = np.zeros((1, g.n_bus))
        p[0, g.from_bus[c]] += 1.0
        p[0, g.to_bus[c]] -= 1.0
        f = dcflow.solve_flows(g.n_bus, g.from_bus.astype(np.int64), g.to_bus.astype(np.int64),
                               g.b, p, g.slack)
        np.testing.assert_allclose(f[0], M[:, c], atol=1e-10)


@pytest.mark.parametrize("seed", [1, 2, 3, 5, 6])
def test_low_rank_split_and_outage_formulas(seed):
    """Brute force vs the rank-k bus-split update and the LODF outage formula,
    restated here in dense FP64:  f' = f0 + W psi,  W = N D S,
    psi = K^-1 (p_M - S^T f0),  K = S^T W,  N' = N - W K^-1 W^T D^-1,
    F^(c) = f' - N'[:,c] f'_c / N'_cc, and N'_cc = 0 exactly for bridges."""
    g = small_grid(seed)
    f0 = dcflow.base_flows(g)
    g = g.with_limits(limits_from_flows(f0[0], 2))
    A, D, X, M = _ptdf_restatement(g)
    N = np.eye(g.n_branch) - M
    f0m = (D @ A @ X @ g.p.T).T
    np.testing.assert_allclose(f0m, f0, atol=1e-10)
    topo = random_topologies(g, 8, seed=seed)
    for gen in topo:
        acts = [a for a in gen if a >= 0]
        k = len(acts)
        S = np.zeros((g.n_branch, k))
        pM = np.zeros((g.T, k))
        for j, a in enumerate(acts):
            s = g.action_station[a]
            bus = g.station_bus[s]
            mask = int(g.action_mask[a])
            for i, e in enumerate(g.station_assets(s)):
                if not (mask >> i) & 1:
                    continue
                if e < 0:
                    pM[:, j] = g.p[:, bus]
                else:
                    S[e, j] = 1.0 if g.from_bus[e] == bus else -1.0
        W = N @ D @ S
        K = S.T @ W
        r = dcflow.evaluate(g, gen, want_flows=True)
        if r["island_base"]:
            assert abs(np.linalg.det(K)) < 1e-8 * max(1.0, np.abs(K).max()) ** k
            continue
        psi = np.linalg.solve(K, (pM - f0 @ S).T)
        fp = f0 + (W @ psi).T
        np.testing.assert_allclose(r["fprime"], fp, atol=1e-9)
        Np = N - W @ np.linalg.solve(K, W.T) @ np.diag(1.0 / g.b)
        for c in range(g.n_branch):
            if c in r["per_outage"]:
                F = fp - np.outer(fp[:, c] / Np[c, c], Np[:, c])
                np.testing.assert_allclose(r["per_outage"][c], F, atol=1e-8)
            else:
                assert abs(Np[c, c]) < 1e-9


def test_metrics_follow_definitions_on_a_random_grid():
    g = small_grid(7, T=3)
    f0 = dcflow.base_flows(g)
    g = g.with_limits(limits_from_flows(f0[0], 3))
    gen = random_topologies(g, 1, seed=3)[0]
    r = dcflow.evaluate(g, gen, want_flows=True)
    assert not r["island_base"]
    lim = g.limit
    fm = np.zeros_like(r["fprime"])
    for F in r["per_outage"].values():
        fm = np.maximum(fm, np.abs(F))
    np.testing.assert_array_equal(fm, r["fmax"])
    lo = sum(max(fm[t, l] - lim[l], 0.0) for t in range(g.T) for l in range(g.n_branch))
    assert r["lambda_o"] == pytest.approx(lo, rel=1e-12)
    ml = max(max(abs(r["fprime"][t, l]), fm[t, l]) / lim[l] for t in range(g.T) for l in range(g.n_branch))
    assert r["maxload"] == pytest.approx(ml, rel=1e-12)
    assert r["fitness"] == pytest.approx(-(lo + ml), rel=1e-12)


def test_descriptors_and_cell():
    g, _ = three_bus()
    a = action_of(g, 0, 2)   # busbar B = {branch 1->2}: 1 moved asset of 3
    assert dcflow.descriptors(g, [a], 8, 8) == (1, 1, 9)
    a = action_of(g, 0, 6)   # B = {branch, injection}: min(1, 2) = 1
    assert dcflow.descriptors(g, [a], 8, 8) == (1, 1, 9)
    assert dcflow.descriptors(g, [-1], 8, 8) == (0, 0, 0)
    big = small_grid(2, n_station=4, k_max=3)
    gen = random_topologies(big, 32, seed=9)
    for row in gen:
        ns, nm, cell = dcflow.descriptors(big, row, 2, 3)
        assert ns == int((row >= 0).sum())
        assert cell == min(ns, 1) * 3 + min(nm, 2)


def test_duplicate_station_rejected():
    g = small_grid(1)
    a0 = int(g.action_offset[0])
    with pytest.raises(dcflow.TopologyError):
        dcflow.evaluate(g.with_limits(np.ones(g.n_branch)), [a0, a0 + 1, -1])


# ----------------------------------------------------------- disconnection slots
def _with_disc(g, disc, n_dslot):
    from dataclasses import replace
    return replace(g, disc=np.array(disc, dtype=np.int32), n_dslot=n_dslot)


def test_disconnection_three_bus_pins():
    """Opening branch 1->2 of the triangle (closed form in the golden fixture):
    the N-0 flows equal that branch's outage, the open branch is no
    contingency, and opening both branches at the slack islands the grid."""
    g, d = three_bus()
    c = d["cases"]["disconnect_1_2"]
    gd = _with_disc(g, [0, 1, 2], 2)
    r = dcflow.evaluate(gd, [-1, 1, -1])
    np.testing.assert_allclose(r["fprime"][0], c["fprime"], atol=1e-12)
    assert r["n_islanded"] == c["n_islanded"] and not r["island_base"]
    for k in ["lambda_o", "maxload", "fitness", "lambda_f1"]:
        assert r[k] == pytest.approx(c[k], abs=1e-12), k
    assert (r["lambda_c"], r["lambda_c0"], r["nd"]) == (c["lambda_c"], c["lambda_c0"], 1)
    r2 = dcflow.evaluate(gd, [-1, 0, 2])
    assert r2["island_base"] and r2["fitness"] == -np.inf
    with pytest.raises(dcflow.TopologyError):
        dcflow.evaluate(gd, [-1, 1, 1])  # one branch opened twice
    with pytest.raises(dcflow.TopologyError):
        dcflow.evaluate(gd, [-1, 3, -1])  # not in the disconnection set


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_disconnection_kirchhoff_and_islanding(seed):
    """With opened branches: KCL and KVL in the N-0 state and every outage
    state, zero flow on opened branches, and islanding equal to networkx's
    connectivity and bridges of the graph without the opened branches."""
    g = small_grid(seed)
    g = _with_disc(g, np.arange(0, g.n_branch, 3), 2).with_limits(np.ones(g.n_branch))
    topo = random_topologies(g, 8, seed=seed)
    assert topo.shape[1] == g.k_max + 2
    seen_open = 0
    for gen in topo:
        opened = dcflow.open_branches(g, gen)
        seen_open += len(opened)
        n_node, fr, to, p, _ = dcflow.post_split_graph(g, gen)
        G = nx.MultiGraph()
        G.add_nodes_from(range(n_node))
        for l in range(len(fr)):
            if l not in opened:
                G.add_edge(int(fr[l]), int(to[l]), key=l)
        r = dcflow.evaluate(g, gen)
        assert r["island_base"] == (not nx.is_connected(G))
        if r["island_base"]:
            continue
        live = np.ones(len(fr), dtype=bool)
        live[opened] = False
        f = dcflow.solve_flows(n_node, fr, to, g.b, p, g.slack, keep=live)
        assert np.all(f[:, opened] == 0.0)
        _kcl_kvl(n_node, fr, to, g.b, p, g.slack, f, skip=-1, opened=opened)
        for c in range(len(fr)):
            if c in opened:
                continue
            keep = live.copy()
            keep[c] = False
            H = G.copy()
            H.remove_edges_from([(u, v, k) for u, v, k in G.edges(keys=True) if k == c])
            if not nx.is_connected(H):
                continue
            F = dcflow.solve_flows(n_node, fr, to, g.b, p, g.slack, keep=keep)
            assert np.all(F[:, c] == 0.0) and np.all(F[:, opened] == 0.0)
            _kcl_kvl(n_node, fr, to, g.b, p, g.slack, F, skip=c, opened=opened)
        bridges = set()
        for u, v, k in G.edges(keys=True):
            H = G.copy()
            H.remove_edge(u, v, key=k)
            if not nx.is_connected(H):
                bridges.add(k)
        n_br = sum(1 for c in g.outages if int(c) in bridges)
        assert r["n_islanded"] == n_br
    assert seen_open > 0


# ------------------------------------------------------------- worst-k export
def test_outage_energy_and_worst_k_three_bus():
    """Per-outage overload energy and the worst-k selection on the triangle,
    from the closed-form outage flows of the golden fixture."""
    g, d = three_bus()
    c = d["cases"]["base"]
    E = dcflow.outage_energy(g, [-1])
    np.testing.assert_allclose(E, c["outage_energy"], atol=1e-12)
    idx, val = dcflow.worst_k(E, 2)
    assert list(idx) == c["worst_2"]
    idx, val = dcflow.worst_k(E, 5)
    assert list(idx) == [1, 0, 2, -1, -1] and np.isnan(val[3:]).all()
    # every outage of the disconnect-1->2 state islands or is the open branch
    gd = _with_disc(g, [0, 1, 2], 2)
    E2 = dcflow.outage_energy(gd, [-1, 1, -1])
    assert np.isnan(E2).all()
    assert list(dcflow.worst_k(E2, 2)[0]) == [-1, -1]


@pytest.mark.parametrize("seed", [1, 2])
def test_outage_energies_sum_like_the_definition(seed):
    """Each N-1 case's energy equals its overloads summed over branches and
    timesteps, recomputed here from networkx-independent re-solves of the
    outage (the plain Laplacian solve with the branch removed)."""
    g = small_grid(seed)
    g = g.with_limits(0.6 * np.abs(dcflow.base_flows(g)).max(axis=0) + 0.05)
    topo = random_topologies(g, 3, seed=seed)
    for gen in topo:
        E = dcflow.outage_energy(g, gen)
        n_node, fr, to, p, _ = dcflow.post_split_graph(g, gen)
        if not dcflow.is_connected_uf(n_node, fr, to):
            assert np.isnan(E).all()
            continue
        L = np.zeros((n_node, n_node))
        for oi, c in enumerate(g.outages):
            if not dcflow.is_connected_uf(n_node, fr, to, skip=int(c)):
                assert np.isnan(E[oi])
                continue
            L[:] = 0.0
            for l in range(len(fr)):
                if l == c:
                    continue
                a, b_ = fr[l], to[l]
                L[a, a] += g.b[l]
                L[b_, b_] += g.b[l]
                L[a, b_] -= g.b[l]
                L[b_, a] -= g.b[l]
            keep = [i for i in range(n_node) if i != g.slack]
            th = np.zeros((p.shape[0], n_node))
            th[:, keep] = np.linalg.solve(L[np.ix_(keep, keep)], p[:, keep].T).T
            F = g.b[None, :] * (th[:, fr] - th[:, to])
            F[:, c] = 0.0
            lim = g.limit[g.monitored]
            ref = np.maximum(np.abs(F[:, g.monitored]) - lim[None, :], 0.0).sum()
            assert E[oi] == pytest.approx(ref, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------- busbar outages
def test_busbar_outages_three_bus():
    g, d = three_bus()
    c = d["cases"]["base"]
    r = dcflow.busbar_outages(g, [-1])
    np.testing.assert_allclose(r["bmax"][0], c["busbar_bmax"], atol=1e-12)
    assert r["lambda_b"] == pytest.approx(c["busbar_lambda_b"], abs=1e-12) and r["n_islanded_busbar"] == 0
    c = d["cases"]["split_branch_and_injection"]
    a = action_of(g, 0, c.get("mask", 6))
    r = dcflow.busbar_outages(g, [a])
    np.testing.assert_allclose(r["bmax"][0], c["busbar_bmax"], atol=1e-12)
    assert r["lambda_b"] == pytest.approx(c["busbar_lambda_b"], abs=1e-12)
    assert r["n_islanded_busbar"] == c["busbar_n_islanded"]
    assert [n for n, _, _ in dcflow.busbar_nodes(g, [a])] == [1, 3]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_busbar_outages_kirchhoff_and_articulation_points(seed):
    """Every busbar outage state obeys KCL and KVL with its node out of
    service, and a busbar outage islands exactly when networkx calls its node
    an articulation point of the topology's graph."""
    g = small_grid(seed)
    g = g.with_limits(np.ones(g.n_branch))
    topo = random_topologies(g, 5, seed=seed)
    for gen in topo:
        n_node, fr, to, p, _ = dcflow.post_split_graph(g, gen)
        if not dcflow.is_connected_uf(n_node, fr, to):
            assert dcflow.busbar_outages(g, gen) is None
            continue
        r = dcflow.busbar_outages(g, gen)
        G = nx.MultiGraph()
        G.add_nodes_from(range(n_node))
        for l in range(len(fr)):
            G.add_edge(int(fr[l]), int(to[l]), key=l)
        art = set(nx.articulation_points(nx.Graph(G)))
        nodes = dcflow.busbar_nodes(g, gen)
        assert r["n_islanded_busbar"] == sum(1 for v, _, _ in nodes if v in art)
        for v, _, _ in nodes:
            if v in art:
                continue
            keep = (fr != v) & (to != v)
            pb = p.copy()
            pb[:, v] = 0.0
            F = dcflow.solve_flows(n_node, fr, to, g.b, pb, g.slack, keep=keep, pin=(v,))
            assert np.all(F[:, ~keep] == 0.0)
            _kcl_kvl(n_node, fr, to, g.b, pb, g.slack, F, opened=list(np.flatnonzero(~keep)))


# ------------------------------------------------------------- lambda_f2 and the lambda_d cell
def _triangle_topology(g, d, name):
    """Genome of a named triangle topology of the golden fixture, on the
    triangle extended with the disconnection set [0, 1, 2] and two slots."""
    gd = _with_disc(g, [0, 1, 2], 2)
    if name.startswith("mask"):
        return gd, [action_of(g, 0, int(name.split()[1])), -1, -1]
    if name == "open 0->2":
        return gd, [-1, 2, -1]
    raise KeyError(name)


def test_lambda_f2_three_bus_hand_values():
    """lambda_f2 with a nonzero busbar penalty Pi(lambda_b - lambda_b^pre) and
    with the penalty clamped at zero, against values derived by hand from the
    triangle's busbar outages (fixture block lambda_f2)."""
    g, d = three_bus()
    for c in d["lambda_f2"]["cases"]:
        gl, gen = _triangle_topology(g.with_limits(np.array(c["limit"])), d, c["topology"])
        pre = dcflow.busbar_outages(gl, [-1, -1, -1])["lambda_b"]
        assert pre == pytest.approx(c["lambda_b_pre"], abs=1e-12)
        r = dcflow.evaluate(gl, gen)
        bb = dcflow.busbar_outages(gl, gen)
        assert bb["lambda_b"] == pytest.approx(c["lambda_b"], abs=1e-12), c
        assert r["lambda_o"] == pytest.approx(c["lambda_o"], abs=1e-12)
        assert (r["lambda_c0"], r["lambda_c"]) == (c["lambda_c0"], c["lambda_c"])
        assert dcflow.lambda_f2(r, bb, pre) == pytest.approx(c["lambda_f2"], abs=1e-12), c
    # a topology that islands the grid has lambda_f2 = -inf
    gl, _ = _triangle_topology(g, d, "mask 6")
    r = dcflow.evaluate(gl, [-1, 0, 2])
    assert r["island_base"] and dcflow.lambda_f2(r, None, 0.0) == -np.inf


def test_cells_with_disconnection_axis_hand_values():
    """Cells of the three-axis archive (split stations, moved assets, opened
    branches), including every clamp at the archive's edge, against values
    derived by hand (fixture block cells_with_disconnections)."""
    g, d = three_bus()
    gd = _with_disc(g, [0, 1, 2], 2)
    for c in d["cells_with_disconnections"]["cases"]:
        split = -1 if c["split"] == "none" else action_of(g, 0, int(c["split"].split()[1]))
        disc = list(c["disc"]) + [-1] * (2 - len(c["disc"]))
        ds, dm, dd = c["extent"]
        ns, nm, cell = dcflow.descriptors(gd, [split] + disc, ds, dm, dd)
        assert (ns, nm, cell) == (c["ns"], c["nm"], c["cell"]), c
        assert len(dcflow.open_branches(gd, [split] + disc)) == c["nd"]
        r = dcflow.evaluate(gd, [split] + disc, d_split=ds, d_moved=dm, d_disc=dd)
        assert r["cell"] == c["cell"] and r["nd"] == c["nd"]


# ------------------------------------------------------------- process-parallel oracle
def _parallel_case(name):
    from dataclasses import replace
    from synth.grids import make_grid
    if name == "300":
        g = make_grid(300, 450, 20, assets=(4, 10), T=3, b_dist=("loguniform", 2.0, 200.0),
                      noise=0.1, seed=11, k_max=4, name="ragged300")
    else:
        from synth import config_grid
        g = config_grid("tto2k")
        # 160 outages, every eighth of them a bridge of the unsplit grid, so that
        # islanding outages fall into several process chunks
        rng = np.random.default_rng(5)
        g = replace(g, outages=np.sort(rng.choice(g.n_branch, 160, replace=False)).astype(np.int32))
    g = g.with_limits(limits_from_flows(dcflow.base_flows(g)[0], max(2, g.n_branch // 100)))
    return g


@pytest.mark.parametrize("name", ["300", "2k"])
def test_parallel_outage_merge_equals_serial(name):
    """The process-parallel oracle (outages split into chunks, maxima merged)
    equals the serial oracle exactly at 2, 3 and 8 processes: the same f^max
    array, islanding count, metrics and per-outage energies, on topologies
    with islanding outages."""
    g = _parallel_case(name)
    topo = random_topologies(g, 6, seed=21)
    seen_isl = 0
    for gen in topo[:3] if name == "2k" else topo:
        ref = dcflow.evaluate(g, gen, want_energy=True)
        for procs in (2, 3, 8):
            r = dcflow.evaluate_parallel_outages(g, gen, processes=procs, want_energy=True)
            assert r["island_base"] == ref["island_base"]
            if ref["island_base"]:
                continue
            assert np.array_equal(r["fmax"], ref["fmax"])
            assert np.array_equal(r["fprime"], ref["fprime"])
            for k in ["n_islanded", "island_any", "lambda_o", "lambda_c", "lambda_c0", "maxload",
                      "fitness", "lambda_f1", "cell"]:
                assert r[k] == ref[k], (k, procs)
            e, e0 = r["outage_energy"], ref["outage_energy"]
            assert np.array_equal(np.isnan(e), np.isnan(e0))
            assert np.array_equal(e[~np.isnan(e)], e0[~np.isnan(e0)])
        seen_isl += int(not ref["island_base"] and ref["n_islanded"] > 0)
    assert seen_isl >= 1
