"""Pins of the MapElites oracle: Philox known-answer vectors, distribution tests
of the mutation draws against scipy's Poisson law and the paper's operation
probabilities, structural invariants of Algorithm 1, and the archive insert
against its definition (best of the batch per cell, first index on ties,
incumbent kept unless strictly beaten)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import mapelites as me
from oracle.philox import philox4x32_10, WordStream, uniform_index
from synth import random_topologies
from tests.gridcases import small_grid, GOLDEN


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert philox4x32_10(r[0:4], r[4:6]) == tuple(r[6:10])


def test_philox_words_uniform():
    ws = WordStream(12345, 7, 3)
    w = np.array([ws.next() for _ in range(40000)], dtype=np.float64)
    hist, _ = np.histogram(w, bins=16, range=(0, 2.0 ** 32))
    chi2 = ((hist - 2500.0) ** 2 / 2500.0).sum()
    assert chi2 < stats.chi2.ppf(0.999, 15)


def test_uniform_index_range_and_balance():
    for n in [1, 2, 3, 7, 1000]:
        assert uniform_index(0, n) == 0
        assert uniform_index(0xFFFFFFFF, n) == n - 1


def test_poisson_thresholds_match_scipy():
    for mean in [0.5, 2.0, 3.7]:
        thr = me.poisson_thresholds(mean, 8)
        ref = [math.floor(stats.poisson.cdf(j, mean) * 2 ** 32) for j in range(8)]
        for a, b in zip(thr, ref):
            assert abs(a - b) <= 2


def test_n_mut_distribution_is_clipped_poisson():
    k = 4
    pthr = me.poisson_thresholds(2.0, k)
    ws = WordStream(99, 0, 0)
    n = 60000
    counts = np.zeros(k + 1)
    for _ in range(n):
        counts[me.draw_n_mut(ws.next(), pthr, k)] += 1
    pmf = stats.poisson.pmf(np.arange(k + 1), 2.0)
    expect = np.zeros(k + 1)
    expect[1] = pmf[0] + pmf[1]
    expect[2:k] = pmf[2:k]
    expect[k] = 1.0 - stats.poisson.cdf(k - 1, 2.0)
    expect *= n
    chi2 = ((counts[1:] - expect[1:]) ** 2 / expect[1:]).sum()
    assert counts[0] == 0
    assert chi2 < stats.chi2.ppf(0.999, k - 1)


@pytest.mark.parametrize("feasible", [0b1111, 0b1110, 0b1101, 0b1001, 0b1000])
def test_operation_draw_follows_renormalised_probabilities(feasible):
    probs = me.DEFAULT_PROBS
    thr = me.op_thresholds(probs, feasible)
    ws = WordStream(5, feasible, 1)
    n = 40000
    counts = np.zeros(4)
    for _ in range(n):
        w = ws.next()
        counts[next(i for i in range(4) if w < thr[i])] += 1
    p = np.array([probs[i] if (feasible >> i) & 1 else 0.0 for i in range(4)])
    p /= p.sum()
    assert np.all(counts[p == 0] == 0)
    e = p[p > 0] * n
    chi2 = ((counts[p > 0] - e) ** 2 / e).sum()
    assert chi2 < stats.chi2.ppf(0.999, max(1, int((p > 0).sum()) - 1))


def test_mutation_invariants():
    g = small_grid(3, n_station=5, k_max=3)
    tab = me.ActionTable(g)
    parents = random_topologies(g, 50, seed=1, min_splits=0)
    for i, par in enumerate(parents):
        for c in range(20):
            ws = WordStream(1, i, c)
            child = me.mutate(par, tab, ws)
            acts = [a for a in child if a >= 0]
            assert len(acts) >= 1
            assert all(0 <= a < g.n_action for a in acts)
            sts = [int(g.action_station[a]) for a in acts]
            assert len(sts) == len(set(sts))
            assert ws.used <= 2 + 3 * 3 + 2


def test_change_keeps_station_and_changes_mask():
    g = small_grid(3, n_station=5, k_max=1)
    tab = me.ActionTable(g)
    a = int(g.action_offset[1]) + 1
    seen_change = 0
    for c in range(400):
        ws = WordStream(3, 0, c)
        child = me.mutate([a], tab, ws, probs=(0.0, 0.0, 1.0, 0.0), mean=1.0)
        assert int(g.action_station[child[0]]) == 1
        assert child[0] != a
        seen_change += 1
    assert seen_change == 400


def test_insert_matches_definition():
    rng = np.random.default_rng(0)
    for trial in range(30):
        arch = me.Archive(4, 4)
        cells0 = rng.integers(0, 16, 6)
        for c in cells0:
            arch.elites[int(c)] = (float(rng.integers(-5, 0)), np.array([int(c)], dtype=np.int32))
        before = dict(arch.elites)
        B = 40
        cells = rng.integers(0, 16, B)
        fit = rng.integers(-6, 1, B).astype(np.float64)
        fit[rng.random(B) < 0.1] = -np.inf
        gens = np.arange(B, dtype=np.int32)[:, None] + 100
        arch.insert(cells, fit, gens)
        for c in range(16):
            idx = [i for i in range(B) if cells[i] == c and np.isfinite(fit[i])]
            if not idx:
                assert arch.elites.get(c) == before.get(c)
                continue
            best = max(fit[i] for i in idx)
            first = min(i for i in idx if fit[i] == best)
            inc = before.get(c)
            if inc is None or best > inc[0]:
                assert arch.elites[c][0] == best and arch.elites[c][1][0] == first + 100
            else:
                assert arch.elites[c] is inc


# ------------------------------------------- disconnection mutation, crossover
def _grid_with_disc(seed=3, n_dslot=2, stride=2):
    from dataclasses import replace
    g = small_grid(seed)
    return replace(g, disc=np.arange(0, g.n_branch, stride, dtype=np.int32), n_dslot=n_dslot)


def test_disconnection_mutation_invariants_and_forced_add():
    g = _grid_with_disc()
    tab = me.ActionTable(g)
    nd = g.n_dslot
    empty = np.full(g.k_max + nd, -1, dtype=np.int32)
    for cand in range(400):
        ws = me.WordStream(5, 1, cand)
        ws.next()
        child = me.mutate(empty, tab, ws, n_dslot=nd, n_disc=g.n_disc)
        d = [x for x in child[g.k_max:] if x >= 0]
        st = [int(tab.station[a]) for a in child[: g.k_max] if a >= 0]
        assert len(set(d)) == len(d) and all(0 <= x < g.n_disc for x in d)
        assert len(set(st)) == len(st)
        assert d or st  # never the unchanged default topology
    # from a genome with all disconnection slots empty and no split, the
    # disconnection step always adds one (the forced rule)
    g1 = _grid_with_disc(n_dslot=1)
    tab1 = me.ActionTable(g1)
    for cand in range(200):
        ws = me.WordStream(9, 2, cand)
        d = [-1]
        me.mutate_disc([-1] * g1.k_max, d, g1.n_disc, ws)
        assert d[0] >= 0


def test_disconnection_operation_frequencies():
    """With every operation feasible, Add / Remove / Change follow 0.25 / 0.25
    / 0.5 and Identity (weight 0) never happens."""
    g = _grid_with_disc(n_dslot=3)
    counts = np.zeros(4)
    base = [0, -1, 5]
    for cand in range(6000):
        ws = me.WordStream(77, 3, cand)
        d = list(base)
        me.mutate_disc([1], d, g.n_disc, ws)
        if d == base:
            counts[me.IDENTITY] += 1
        elif sum(x >= 0 for x in d) == 3:
            counts[me.ADD] += 1
        elif sum(x >= 0 for x in d) == 1:
            counts[me.REMOVE] += 1
        else:
            counts[me.CHANGE] += 1
    assert counts[me.IDENTITY] == 0
    exp = 6000 * np.array([0.25, 0.25, 0.5])
    chi2 = (((counts[:3] - exp) ** 2) / exp).sum()
    assert chi2 < stats.chi2.ppf(0.999, 2)


def test_crossover_definition():
    """p_c1 = 1 reproduces parent 1; children draw only from the parents'
    union with distinct stations and branches; with disjoint parents and
    p_c1 = 0.5 the first slot comes from parent 1 half of the time."""
    g = _grid_with_disc(n_dslot=2)
    tab = me.ActionTable(g)
    topo = random_topologies(g, 64, seed=4)
    from1 = 0
    trials = 0
    for i in range(0, 64, 2):
        p1, p2 = topo[i], topo[i + 1]
        for cand in range(40):
            ws = me.WordStream(3, i, cand)
            c = me.crossover(p1, p2, tab, ws, n_dslot=2, p_c1=1.0)
            assert set(x for x in c[: g.k_max] if x >= 0) == set(x for x in p1[: g.k_max] if x >= 0)
            assert set(x for x in c[g.k_max:] if x >= 0) == set(x for x in p1[g.k_max:] if x >= 0)
            ws = me.WordStream(4, i, cand)
            c = me.crossover(p1, p2, tab, ws, n_dslot=2, p_c1=0.5)
            acts = [int(x) for x in c[: g.k_max] if x >= 0]
            dis = [int(x) for x in c[g.k_max:] if x >= 0]
            assert set(acts) <= set(int(x) for x in np.concatenate([p1[: g.k_max], p2[: g.k_max]]) if x >= 0)
            assert set(dis) <= set(int(x) for x in np.concatenate([p1[g.k_max:], p2[g.k_max:]]) if x >= 0)
            assert len({int(tab.station[a]) for a in acts}) == len(acts)
            assert len(set(dis)) == len(dis)
            s1 = {int(tab.station[a]) for a in p1[: g.k_max] if a >= 0}
            s2 = {int(tab.station[a]) for a in p2[: g.k_max] if a >= 0}
            if s1 and s2 and not (s1 & s2) and acts:
                trials += 1
                from1 += int(tab.station[acts[0]]) in s1
    assert trials > 200
    assert abs(from1 / trials - 0.5) < 4 * math.sqrt(0.25 / trials)


def test_mutation_crossover_split_is_uniform():
    B = 10
    counts = np.zeros(B + 1)
    for it in range(5500):
        counts[me.mutation_count(11, it, B, True)] += 1
    assert me.mutation_count(11, 0, B, False) == B
    exp = 5500 / (B + 1)
    chi2 = (((counts - exp) ** 2) / exp).sum()
    assert chi2 < stats.chi2.ppf(0.999, B)
