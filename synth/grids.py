"""Synthetic transmission grids, station action tables and evaluation batches.

Every function here is seeded and deterministic.  The recipe stands in for the
proprietary TSO grids of the paper (Table 1) and follows the workload shapes of
the DC N-1 topology search: a meshed planar-like graph (random spanning tree plus
short extra edges), a north/south injection imbalance that loads the grid,
thermal limits derived from base-case flows with a few tightened branches, and
substations whose assets (incident branches plus one injection) can be split
onto two busbars (two-node operation, Sec. "Switching actions").

Nothing in this module solves a loadflow.  Thermal limits are produced by
:func:`limits_from_flows` from base flows that the caller computed elsewhere.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np
from scipy.spatial import cKDTree

INJECTION = -1  # asset code for a station's injection


@dataclass
class SynthGrid:
    """A bus/branch grid plus its splittable stations and action set.

    Arrays use the layouts passed across the library boundary:
    ``from_bus``/``to_bus`` int32 [E], ``b`` float64 [E] (p.u. susceptance),
    ``p`` float64 [T][n_bus] (the slack entry balances each timestep),
    ``limit`` float64 [E] or None, ``monitored`` / ``outages`` int32 branch ids,
    stations as CSR (``asset_offset`` [S+1], ``asset_branch`` with -1 for the
    injection), actions grouped by station (``action_offset`` [S+1],
    ``action_station`` [A], ``action_mask`` uint32 [A], bit i set = asset i on
    busbar B; asset 0 always stays on busbar A).  ``disc`` int32 is the
    disconnection set (branch ids that a genome may open) and ``n_dslot`` the
    number of disconnection slots that follow the ``k_max`` split slots in a
    genome (Sec. "Repertoire design": N_a split slots, N_d disconnection slots).
    """

    name: str
    n_bus: int
    from_bus: np.ndarray
    to_bus: np.ndarray
    b: np.ndarray
    slack: int
    p: np.ndarray
    limit: np.ndarray | None
    monitored: np.ndarray
    outages: np.ndarray
    station_bus: np.ndarray
    asset_offset: np.ndarray
    asset_branch: np.ndarray
    action_offset: np.ndarray
    action_station: np.ndarray
    action_mask: np.ndarray
    k_max: int
    xy: np.ndarray = field(repr=False, default=None)
    seed: int = 0
    disc: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    n_dslot: int = 0

    @property
    def n_branch(self) -> int:
        return int(self.from_bus.shape[0])

    @property
    def T(self) -> int:
        return int(self.p.shape[0])

    @property
    def n_station(self) -> int:
        return int(self.station_bus.shape[0])

    @property
    def n_action(self) -> int:
        return int(self.action_station.shape[0])

    @property
    def n_disc(self) -> int:
        return int(self.disc.shape[0])

    @property
    def genome_width(self) -> int:
        return self.k_max + self.n_dslot

    def with_limits(self, limit: np.ndarray) -> "SynthGrid":
        return replace(self, limit=np.ascontiguousarray(limit, dtype=np.float64))

    def station_assets(self, s: int) -> np.ndarray:
        return self.asset_branch[self.asset_offset[s]:self.asset_offset[s + 1]]


class _DSU:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        p = self.p
        while p[x] != x:
            p[x] = p[p[x]]
            x = p[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return False
        self.p[rb] = ra
        return True


def _spanning_tree_plus_extras(xy, n_branch, rng, knn=6):
    """Random-weight Kruskal tree over a k-nearest-neighbour graph plus the
    shortest remaining candidate edges.  Returns (edges [E][2], is_tree [E])."""
    n = xy.shape[0]
    kd = cKDTree(xy)
    k = min(knn + 1, n)
    _, idx = kd.query(xy, k=k)
    cand = set()
    for i in range(n):
        for j in idx[i, 1:]:
            j = int(j)
            if i != j:
                cand.add((min(i, j), max(i, j)))
    cand = sorted(cand)
    w = rng.random(len(cand))
    dsu = _DSU(n)
    tree = []
    for e in np.argsort(w, kind="stable"):
        a, b2 = cand[e]
        if dsu.union(a, b2):
            tree.append((a, b2))
    # the k-NN graph can leave separate clusters: join each to its nearest
    # point outside the cluster until the tree spans all buses
    while len(tree) < n - 1:
        roots = np.array([dsu.find(i) for i in range(n)])
        main = roots[0]
        other = np.flatnonzero(roots != main)
        inside = np.flatnonzero(roots == main)
        kd_in = cKDTree(xy[inside])
        d, j = kd_in.query(xy[other])
        o = int(other[int(np.argmin(d))])
        m = int(inside[int(j[int(np.argmin(d))])])
        dsu.union(m, o)
        tree.append((min(m, o), max(m, o)))
    tree_set = set(tree)
    n_extra = n_branch - (n - 1)
    if n_extra < 0:
        raise ValueError("n_branch must be at least n_bus - 1")
    rest = [e for e in cand if e not in tree_set]
    length = np.array([np.hypot(*(xy[a] - xy[b2])) for a, b2 in rest]) if rest else np.zeros(0)
    order = np.argsort(length, kind="stable")
    if len(rest) < n_extra:
        raise ValueError("not enough candidate edges for the requested branch count")
    extra = [rest[i] for i in order[:n_extra]]
    edges = tree + extra
    is_tree = np.array([True] * len(tree) + [False] * len(extra))
    return edges, is_tree


def _non_bridge_mask(n, edges, is_tree):
    """Branches that lie on a cycle, from the construction itself: every extra
    edge closes a cycle with the tree path between its ends, so those tree
    edges are covered.  Covered tree edges are contracted as they are found so
    each is visited once."""
    E = len(edges)
    adj = [[] for _ in range(n)]
    for e, (a, b2) in enumerate(edges):
        if is_tree[e]:
            adj[a].append((b2, e))
            adj[b2].append((a, e))
    parent = [-1] * n
    pedge = [-1] * n
    depth = [0] * n
    seen = [False] * n
    seen[0] = True
    stack = [0]
    while stack:
        u = stack.pop()
        for v, e in adj[u]:
            if not seen[v]:
                seen[v] = True
                parent[v] = u
                pedge[v] = e
                depth[v] = depth[u] + 1
                stack.append(v)
    up = list(range(n))  # contracted "representative" pointer

    def top(x):
        while up[x] != x:
            up[x] = up[up[x]]
            x = up[x]
        return x

    covered = np.zeros(E, dtype=bool)
    for e, (a, b2) in enumerate(edges):
        if is_tree[e]:
            continue
        covered[e] = True
        u, v = top(a), top(b2)
        while u != v:
            if depth[u] < depth[v]:
                u, v = v, u
            covered[pedge[u]] = True
            up[u] = top(parent[u])
            u = up[u]
    return covered


def make_grid(n_bus: int, n_branch: int, n_station: int, assets=(4, 6), T: int = 1,
              b_dist=("uniform", 5.0, 50.0), noise: float = 0.0, seed: int = 0,
              n_outage: int | None = None, k_max: int = 2, name: str = "grid",
              knn: int = 6, n_disc: int = 0, n_dslot: int = 0) -> SynthGrid:
    """Build a synthetic grid (limits left unset; see :func:`limits_from_flows`).
    ``n_disc`` non-bridge branches form the disconnection set (drawn from a
    separate stream, so the rest of the grid does not depend on it)."""
    rng = np.random.default_rng(seed)
    xy = rng.random((n_bus, 2))
    edges, is_tree = _spanning_tree_plus_extras(xy, n_branch, rng, knn=knn)
    E = len(edges)
    flip = rng.random(E) < 0.5
    fr = np.array([b2 if f else a for (a, b2), f in zip(edges, flip)], dtype=np.int32)
    to = np.array([a if f else b2 for (a, b2), f in zip(edges, flip)], dtype=np.int32)
    kind, lo, hi = b_dist
    if kind == "uniform":
        b = rng.uniform(lo, hi, E)
    elif kind == "loguniform":
        b = np.exp(rng.uniform(math.log(lo), math.log(hi), E))
    else:
        raise ValueError(kind)
    slack = int(np.argmin(np.hypot(xy[:, 0] - 0.5, xy[:, 1] - 0.5)))

    # north/south imbalance: 8 of 30 buses on each side, scaled with n
    n_ns = max(1, int(round(n_bus * 8 / 30)))
    by_y = np.argsort(xy[:, 1], kind="stable")
    south = by_y[:n_ns]
    north = by_y[-n_ns:]
    base = np.zeros(n_bus)
    base[north] = rng.normal(1.0, 0.3, n_ns)
    base[south] = -rng.normal(1.0, 0.3, n_ns)
    p = np.tile(base, (T, 1))
    if noise > 0:
        p = p + rng.normal(0.0, noise, (T, n_bus))
    others = np.ones(n_bus, dtype=bool)
    others[slack] = False
    p[:, slack] = -p[:, others].sum(axis=1)

    # splittable stations: non-slack buses whose branch count fits the asset range
    deg = np.bincount(np.concatenate([fr, to]), minlength=n_bus)
    amin, amax = assets
    eligible = np.flatnonzero((deg >= max(3, amin - 1)) & (deg + 1 <= amax) & others)
    if eligible.size < n_station:
        raise ValueError(f"only {eligible.size} eligible stations for {n_station} requested")
    st = np.sort(rng.choice(eligible, n_station, replace=False)).astype(np.int32)
    inc = [[] for _ in range(n_bus)]
    for e in range(E):
        inc[fr[e]].append(e)
        inc[to[e]].append(e)
    a_off = [0]
    a_br = []
    act_off = [0]
    act_st = []
    act_mask = []
    for s_i, s in enumerate(st):
        lst = sorted(inc[s]) + [INJECTION]
        a_br.extend(lst)
        a_off.append(len(a_br))
        m = len(lst)
        is_branch = np.array([x >= 0 for x in lst])
        for mm in range(1, 1 << (m - 1)):
            mask = mm << 1  # asset 0 stays on busbar A
            onb = np.array([(mask >> i) & 1 for i in range(m)], dtype=bool)
            if not (onb & is_branch).any():
                continue  # busbar B without a branch
            act_st.append(s_i)
            act_mask.append(mask)
        act_off.append(len(act_st))

    nb_mask = None
    if n_outage is None:
        outages = np.arange(E, dtype=np.int32)
    else:
        nb_mask = _non_bridge_mask(n_bus, edges, is_tree)
        nb = np.flatnonzero(nb_mask)
        if nb.size < n_outage:
            raise ValueError("not enough non-bridge branches for the outage set")
        outages = np.sort(rng.choice(nb, n_outage, replace=False)).astype(np.int32)
    disc = np.zeros(0, dtype=np.int32)
    if n_disc > 0:
        if nb_mask is None:
            nb_mask = _non_bridge_mask(n_bus, edges, is_tree)
        nb = np.flatnonzero(nb_mask)
        if nb.size < n_disc:
            raise ValueError("not enough non-bridge branches for the disconnection set")
        disc = np.sort(np.random.default_rng(seed + 31337).choice(nb, n_disc, replace=False)).astype(np.int32)
    return SynthGrid(
        name=name, n_bus=n_bus, from_bus=fr, to_bus=to, b=b.astype(np.float64), slack=slack,
        p=np.ascontiguousarray(p, dtype=np.float64), limit=None,
        monitored=np.arange(E, dtype=np.int32), outages=outages,
        station_bus=st, asset_offset=np.array(a_off, dtype=np.int32),
        asset_branch=np.array(a_br, dtype=np.int32),
        action_offset=np.array(act_off, dtype=np.int32),
        action_station=np.array(act_st, dtype=np.int32),
        action_mask=np.array(act_mask, dtype=np.uint32), k_max=k_max, xy=xy, seed=seed,
        disc=disc, n_dslot=int(n_dslot))


def limits_from_flows(f0_t0: np.ndarray, n_tight: int, seed: int = 0) -> np.ndarray:
    """Thermal limits from base-case flows of the unsplit grid at t = 0:
    1.1 |f0| + 0.1, with ``n_tight`` branches of above-median |f0| tightened
    to 0.8x so that the base case carries overloads."""
    rng = np.random.default_rng(seed + 7919)
    a = np.abs(np.asarray(f0_t0, dtype=np.float64))
    lim = 1.1 * a + 0.1
    cand = np.flatnonzero(a > np.median(a))
    if n_tight > 0 and cand.size:
        pick = rng.choice(cand, min(n_tight, cand.size), replace=False)
        lim[pick] *= 0.8
    return lim


def random_topologies(grid: SynthGrid, B: int, k_max: int | None = None, seed: int = 0,
                      min_splits: int = 1) -> np.ndarray:
    """B genomes of ``k_max`` action slots (-1 = empty): the number of splits is
    uniform in [min_splits, k_max], stations are distinct, and each station's
    action is uniform over its action list.  A grid with disconnection slots
    appends ``n_dslot`` of them: the number of disconnections is uniform in
    [0, n_dslot], the branches distinct and uniform over the disconnection set."""
    k_max = grid.k_max if k_max is None else k_max
    rng = np.random.default_rng(seed + 104729)
    S = grid.n_station
    kk = min(k_max, S)
    ns = rng.integers(min_splits, kk + 1, size=B)
    out = np.full((B, k_max), -1, dtype=np.int32)
    off = grid.action_offset
    cnt = np.diff(off)
    chunk = max(1, (1 << 22) // max(S, 1))
    for s0 in range(0, B, chunk):
        s1 = min(B, s0 + chunk)
        keys = rng.random((s1 - s0, S))
        sta = np.argpartition(keys, kk - 1, axis=1)[:, :kk] if kk < S else np.argsort(keys, axis=1)
        r = rng.random((s1 - s0, kk))
        act = off[sta] + np.minimum((r * cnt[sta]).astype(np.int64), cnt[sta] - 1)
        for j in range(kk):
            sel = ns[s0:s1] > j
            out[s0:s1, j] = np.where(sel, act[:, j], -1)
    if grid.n_dslot > 0 and grid.n_disc > 0:
        drng = np.random.default_rng(seed + 7777)
        nd_max = min(grid.n_dslot, grid.n_disc)
        nd = drng.integers(0, nd_max + 1, size=B)
        dpart = np.full((B, grid.n_dslot), -1, dtype=np.int32)
        keys = drng.random((B, grid.n_disc))
        pick = np.argsort(keys, axis=1)[:, :nd_max]
        for j in range(nd_max):
            dpart[:, j] = np.where(nd > j, pick[:, j], -1)
        out = np.concatenate([out, dpart], axis=1)
    elif grid.n_dslot > 0:
        out = np.concatenate([out, np.full((B, grid.n_dslot), -1, dtype=np.int32)], axis=1)
    return out


# Workload recipes.  The 30-bus branch count reads "spanning tree plus extra
# edges, 41 branches" as 29 + 12 = 41.
CONFIGS = {
    "tto30": dict(n_bus=30, n_branch=41, n_station=6, assets=(4, 6), T=1,
                  b_dist=("uniform", 5.0, 50.0), noise=0.0, n_outage=None, k_max=2,
                  n_tight=5, batch=256, archive=(8, 8), iterations=20),
    "tto2k": dict(n_bus=2000, n_branch=3000, n_station=150, assets=(4, 10), T=16,
                  b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=None, k_max=4,
                  n_tight=30, batch=4096, archive=(8, 8), iterations=20),
    "tto10k": dict(n_bus=10000, n_branch=15000, n_station=400, assets=(4, 10), T=4,
                   b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=5000, k_max=6,
                   n_tight=150, batch=8192, archive=(20, 20), iterations=1000),
    # mixed-size members of the one-launch batching workload (the two large grids
    # sample a third of their branches as outages, like the 10000-bus workload)
    "mix500": dict(n_bus=500, n_branch=750, n_station=40, assets=(4, 10), T=1,
                   b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=None, k_max=4,
                   n_tight=8, batch=1024, archive=(8, 8), iterations=20),
    "mix2k": dict(n_bus=2000, n_branch=3000, n_station=150, assets=(4, 10), T=4,
                  b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=None, k_max=4,
                  n_tight=30, batch=2048, archive=(8, 8), iterations=20),
    "mix5k": dict(n_bus=5000, n_branch=7500, n_station=250, assets=(4, 10), T=16,
                  b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=2500, k_max=4,
                  n_tight=75, batch=4096, archive=(8, 8), iterations=20),
    "mix10k": dict(n_bus=10000, n_branch=15000, n_station=400, assets=(4, 10), T=24,
                   b_dist=("loguniform", 2.0, 200.0), noise=0.1, n_outage=5000, k_max=4,
                   n_tight=150, batch=8192, archive=(8, 8), iterations=20),
}


def config_grid(name: str, seed: int = 0, **overrides) -> SynthGrid:
    """The grid of a named workload recipe, limits still unset."""
    c = dict(CONFIGS[name])
    c.update(overrides)
    return make_grid(c["n_bus"], c["n_branch"], c["n_station"], assets=c["assets"], T=c["T"],
                     b_dist=c["b_dist"], noise=c["noise"], seed=seed, n_outage=c["n_outage"],
                     k_max=c["k_max"], name=name, n_disc=c.get("n_disc", 0), n_dslot=c.get("n_dslot", 0))
