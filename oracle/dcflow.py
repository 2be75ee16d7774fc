"""Brute-force FP64 DC N-1 evaluation of split topologies (test oracle).

For every candidate topology the oracle builds the post-split bus/branch graph,
solves the DC loadflow from scratch, and re-solves the whole grid once per
outage with that branch removed.  No PTDF, LODF or low-rank update is used:
these are the plain definitions that the fast path must reproduce.

Definitions followed:
  * DC flows f_l = b_l (theta_from - theta_to) with B theta = p, slack angle 0
    (Sec. "Importer": linearised DC representation).
  * Two-node operation of a split station (Sec. "Switching actions"): the assets
    on busbar B move to a new node; busbar A keeps the rest.
  * f_e^max = max over outages of |f_e^(o)| (Sec. "Fitness function heuristics").
  * lambda_o = sum_e Pi(f_e^max - fbar_e), lambda_c = sum_e 1(f_e^max > fbar_e),
    lambda_c0 = sum_e 1(|f_e^n0| > fbar_e) (same section).
  * lambda_f1 = -(lambda_o + 200 lambda_c0 + 50 lambda_c) (Sec. "High-level
    Genetic Algorithm loop").
  * Workload fitness = -(lambda_o + max loading), max loading over N-0 and N-1.
  * lambda_s = number of split stations; lambda_r read as the number of moved
    assets min(|A|, |B|) per split (Sec. "Fitness function heuristics",
    "Repertoire design").

Readings where the paper is silent (each also listed in the design notes):
  * an outage that islands the post-split grid is skipped in the maximum and
    counted; a topology whose split itself islands the grid is invalid
    (fitness -inf);
  * with several timesteps, lambda_o / lambda_c / lambda_c0 sum over timesteps
    and max loading takes the maximum over timesteps;
  * cell = min(lambda_s, D_s - 1) * D_m + min(moved, D_m - 1), times D_d plus
    min(lambda_d, D_d - 1) when the archive also spans disconnections;
  * disconnection slots (Sec. "Repertoire design": a genome holds N_a split
    slots and N_d disconnection slots) open their branch in every state; an
    outage of a branch the topology already opened is no contingency and is
    skipped without counting as islanding; a split whose busbar B keeps only
    opened branches leaves its new node isolated, which islands the grid.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

DENSE_MAX = 64


class TopologyError(ValueError):
    pass


def _find(parent, x):
    while parent[x] != x:
        parent[x] = parent[parent[x]]
        x = parent[x]
    return x


def is_connected_uf(n_node, fr, to, skip=-1):
    """Union-find connectivity over all nodes (an isolated node counts)."""
    parent = list(range(n_node))
    comps = n_node
    for e in range(len(fr)):
        if e == skip:
            continue
        a, b = _find(parent, int(fr[e])), _find(parent, int(to[e]))
        if a != b:
            parent[b] = a
            comps -= 1
    return comps == 1


def _is_connected_cs(n_node, fr, to, keep):
    g = sp.coo_matrix((np.ones(int(keep.sum())), (fr[keep], to[keep])), shape=(n_node, n_node))
    nc, _ = csg.connected_components(g, directed=False)
    return nc == 1


def split_part(grid, genome):
    """The split slots of a genome: all of it for a grid without disconnection
    slots, else its first k_max entries."""
    return list(genome) if getattr(grid, "n_dslot", 0) == 0 else list(genome)[: grid.k_max]


def open_branches(grid, genome):
    """Sorted branch ids opened by the disconnection slots of ``genome``
    (indices into the grid's disconnection set, -1 = empty)."""
    nd = getattr(grid, "n_dslot", 0)
    if nd == 0:
        return []
    out = []
    for d in list(genome)[grid.k_max: grid.k_max + nd]:
        d = int(d)
        if d < 0:
            continue
        if d >= grid.n_disc:
            raise TopologyError(f"unknown disconnection {d}")
        e = int(grid.disc[d])
        if e in out:
            raise TopologyError(f"branch {e} opened twice")
        out.append(e)
    return sorted(out)


def post_split_graph(grid, genome):
    """Apply the split actions of ``genome`` (action ids, -1 = empty slot).

    Returns (n_node, from', to', p' [T][n_node], slots) where each split slot j
    adds node n_bus + j holding the assets of busbar B.  ``slots`` lists
    (station, mask, n_assets) for the descriptors.
    """
    fr = grid.from_bus.astype(np.int64).copy()
    to = grid.to_bus.astype(np.int64).copy()
    n = grid.n_bus
    acts = [int(a) for a in split_part(grid, genome) if int(a) >= 0]
    seen = set()
    slots = []
    for a in acts:
        if a >= grid.n_action:
            raise TopologyError(f"unknown action id {a}")
        s = int(grid.action_station[a])
        if s in seen:
            raise TopologyError(f"station {s} split twice")
        seen.add(s)
        slots.append((s, int(grid.action_mask[a]), int(grid.asset_offset[s + 1] - grid.asset_offset[s])))
    n_node = n + len(slots)
    p = np.zeros((grid.T, n_node))
    p[:, :n] = grid.p
    for j, (s, mask, m) in enumerate(slots):
        bus = int(grid.station_bus[s])
        node = n + j
        assets = grid.station_assets(s)
        for i in range(m):
            if not (mask >> i) & 1:
                continue
            e = int(assets[i])
            if e < 0:
                p[:, node] = p[:, bus]
                p[:, bus] = 0.0
            elif fr[e] == bus:
                fr[e] = node
            elif to[e] == bus:
                to[e] = node
            else:
                raise TopologyError("asset branch not incident to its station")
    return n_node, fr, to, p, slots


def solve_flows(n_node, fr, to, b, p, slack, skip=-1, keep=None, pin=()):
    """DC loadflow: branch flows [T][E] for injections p [T][n_node]; branch
    ``skip`` and the branches outside ``keep`` are out of service (flow 0).  The
    slack angle is fixed at 0 and the slack absorbs any imbalance.  Nodes in
    ``pin`` (isolated, without injection) get angle 0."""
    E = len(fr)
    keep = np.ones(E, dtype=bool) if keep is None else np.array(keep, dtype=bool)
    if skip >= 0:
        keep[skip] = False
    f, t, w = fr[keep], to[keep], b[keep]
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([w, w, -w, -w])
    if pin:
        rows = np.concatenate([rows, np.asarray(pin, dtype=rows.dtype)])
        cols = np.concatenate([cols, np.asarray(pin, dtype=cols.dtype)])
        vals = np.concatenate([vals, np.ones(len(pin))])
    L = sp.coo_matrix((vals, (rows, cols)), shape=(n_node, n_node)).tocsc()
    idx = np.array([i for i in range(n_node) if i != slack])
    Lr = L[idx][:, idx]
    rhs = p[:, idx].T
    if n_node <= DENSE_MAX:
        th_r = np.linalg.solve(Lr.toarray(), rhs)
    else:
        th_r = spla.splu(Lr.tocsc()).solve(np.ascontiguousarray(rhs))
    theta = np.zeros((n_node, p.shape[0]))
    theta[idx] = th_r.reshape(len(idx), -1)
    flows = b[:, None] * (theta[fr] - theta[to])
    flows[~keep] = 0.0
    return flows.T


def base_flows(grid):
    """Flows [T][E] of the unsplit grid."""
    return solve_flows(grid.n_bus, grid.from_bus.astype(np.int64), grid.to_bus.astype(np.int64),
                       grid.b, grid.p, grid.slack)


def descriptors(grid, genome, d_split, d_moved, d_disc=1):
    """(lambda_s, moved assets, cell) of a genome; with d_disc > 1 the cell
    also spans lambda_d, the number of opened branches."""
    ns = 0
    nm = 0
    for a in split_part(grid, genome):
        a = int(a)
        if a < 0:
            continue
        s = int(grid.action_station[a])
        m = int(grid.asset_offset[s + 1] - grid.asset_offset[s])
        on_b = bin(int(grid.action_mask[a])).count("1")
        ns += 1
        nm += min(on_b, m - on_b)
    cell = min(ns, d_split - 1) * d_moved + min(nm, d_moved - 1)
    if d_disc > 1:
        cell = cell * d_disc + min(len(open_branches(grid, genome)), d_disc - 1)
    return ns, nm, cell


def evaluate(grid, genome, timesteps=None, outages=None, d_split=8, d_moved=8, want_flows=False, d_disc=1,
             want_energy=False):
    """Evaluate one topology by brute force.

    ``outages`` optionally restricts the outage list (indices into
    ``grid.outages``) for sampled checks; the default is the full set.
    Returns a dict with the islanding flags, f' (N-0 flows of monitored
    branches) [T][E_mon], fmax [T][E_mon], the metrics, fitness and cell.
    """
    tsel = np.arange(grid.T) if timesteps is None else np.asarray(timesteps)
    n_node, fr, to, p, _ = post_split_graph(grid, genome)
    opened = open_branches(grid, genome)
    live = np.ones(len(fr), dtype=bool)
    live[opened] = False
    p = p[tsel]
    ns, nm, cell = descriptors(grid, genome, d_split, d_moved, d_disc)
    mon = grid.monitored.astype(np.int64)
    lim = grid.limit[mon]
    res = dict(ns=ns, nm=nm, nd=len(opened), cell=cell)
    if not (is_connected_uf(n_node, fr, to) if not opened else _is_connected_cs(n_node, fr, to, live)):
        res.update(island_base=True, island_any=False, n_islanded=0, fitness=-np.inf,
                   lambda_f1=-np.inf)
        return res
    f_n0 = solve_flows(n_node, fr, to, grid.b, p, grid.slack, keep=live)
    fprime = f_n0[:, mon]
    out_idx = np.arange(grid.outages.size) if outages is None else np.asarray(outages)
    fmax = np.zeros_like(fprime)
    n_isl = 0
    per_outage = {} if want_flows else None
    energy = np.full(grid.outages.size, np.nan) if want_energy else None
    for oi in out_idx:
        c = int(grid.outages[oi])
        if not live[c]:
            continue  # already open: no contingency
        keep = live.copy()
        keep[c] = False
        if not _is_connected_cs(n_node, fr, to, keep):
            n_isl += 1
            continue
        F = solve_flows(n_node, fr, to, grid.b, p, grid.slack, keep=keep)[:, mon]
        if want_flows:
            per_outage[int(oi)] = F
        if want_energy:
            energy[oi] = float(np.maximum(np.abs(F) - lim[None, :], 0.0).sum())
        fmax = np.maximum(fmax, np.abs(F))
    over = np.maximum(fmax - lim[None, :], 0.0)
    lam_o = float(over.sum())
    lam_c = int((fmax > lim[None, :]).sum())
    lam_c0 = int((np.abs(fprime) > lim[None, :]).sum())
    maxload = float(np.max(np.maximum(np.abs(fprime), fmax) / lim[None, :]))
    res.update(island_base=False, island_any=n_isl > 0, n_islanded=n_isl, fprime=fprime,
               fmax=fmax, lambda_o=lam_o, lambda_c=lam_c, lambda_c0=lam_c0, maxload=maxload,
               fitness=-(lam_o + maxload), lambda_f1=-(lam_o + 200.0 * lam_c0 + 50.0 * lam_c))
    if want_flows:
        res["per_outage"] = per_outage
    if want_energy:
        res["outage_energy"] = energy
    return res


def busbar_nodes(grid, genome):
    """The busbar outage set O_b of a topology (reading): every splittable
    station's node, and for a split station both its nodes (busbar A keeps the
    station bus, busbar B is the new node).  Returns (node, station, side)."""
    _, _, _, _, slots = post_split_graph(grid, genome)
    split_node = {s: grid.n_bus + j for j, (s, _, _) in enumerate(slots)}
    out = []
    for s in range(grid.n_station):
        out.append((int(grid.station_bus[s]), s, 0))
        if s in split_node:
            out.append((split_node[s], s, 1))
    return out


def busbar_outages(grid, genome, timesteps=None):
    """Busbar outages of one topology by brute force (Sec. "Fitness function
    heuristics": lambda_b = sum_e Pi(max_b |f_e^(b)| - fbar_e)).  A busbar
    outage takes its node out of service: every branch at the node opens and
    its injection is lost (the slack balances).  When the rest of the grid
    falls apart the outage islands: it is skipped and counted.  Returns bmax
    [T][E_mon] (max over busbar outages of |flow|), the islanding count and
    lambda_b (summed over timesteps like lambda_o); None for a topology that
    islands the grid."""
    tsel = np.arange(grid.T) if timesteps is None else np.asarray(timesteps)
    n_node, fr, to, p, _ = post_split_graph(grid, genome)
    opened = open_branches(grid, genome)
    live = np.ones(len(fr), dtype=bool)
    live[opened] = False
    p = p[tsel]
    if not _is_connected_cs(n_node, fr, to, live):
        return None
    mon = grid.monitored.astype(np.int64)
    lim = grid.limit[mon]
    bmax = np.zeros((len(tsel), mon.size))
    n_isl = 0
    for v, _, _ in busbar_nodes(grid, genome):
        keep = live & (fr != v) & (to != v)
        g = sp.coo_matrix((np.ones(int(keep.sum())), (fr[keep], to[keep])), shape=(n_node, n_node))
        _, lab = csg.connected_components(g, directed=False)
        rest = np.delete(lab, v)
        if np.any(rest != rest[0]):
            n_isl += 1
            continue
        pb = p.copy()
        pb[:, v] = 0.0
        F = solve_flows(n_node, fr, to, grid.b, pb, grid.slack, keep=keep, pin=(v,))
        bmax = np.maximum(bmax, np.abs(F[:, mon]))
    return dict(bmax=bmax, n_islanded_busbar=n_isl,
                lambda_b=float(np.maximum(bmax - lim[None, :], 0.0).sum()))


def lambda_f2(res, busbar, lambda_b_pre):
    """lambda_f2 = -(lambda_o + 200 lambda_c0 + 50 lambda_c + Pi(lambda_b -
    lambda_b^pre)) (Sec. "High-level Genetic Algorithm loop"); -inf for a
    topology that islands the grid."""
    if res["island_base"]:
        return -np.inf
    return -(res["lambda_o"] + 200.0 * res["lambda_c0"] + 50.0 * res["lambda_c"]
             + max(busbar["lambda_b"] - lambda_b_pre, 0.0))


def outage_energy(grid, genome, timesteps=None):
    """Overload energy of every N-1 case of one topology (Sec. "AC-Validator":
    the DC optimiser computes each N-1 case's overload energy to pick the worst
    k): E_c = sum over timesteps and monitored branches of max(|F_l^(c)| -
    fbar_l, 0).  NaN for an outage that islands the topology or whose branch it
    already opened; all NaN when the topology itself islands the grid."""
    r = evaluate(grid, genome, timesteps=timesteps, want_energy=True)
    if r["island_base"]:
        return np.full(grid.outages.size, np.nan)
    return r["outage_energy"]


def worst_k(energy, k):
    """The k outages (indices into the outage list) of largest overload energy,
    larger energy first and the lower index first among equal energies; NaN
    entries never qualify.  Returns (indices, energies), padded with -1 / NaN."""
    e = np.asarray(energy, dtype=np.float64)
    ok = np.flatnonzero(~np.isnan(e))
    order = ok[np.lexsort((ok, -e[ok]))][:k]
    idx = np.full(k, -1, dtype=np.int64)
    val = np.full(k, np.nan)
    idx[: order.size] = order
    val[: order.size] = e[order]
    return idx, val


def _pool(processes):
    """A spawn-started process pool whose workers run single-threaded BLAS
    (one solve per process; threaded BLAS in every worker oversubscribes the
    host)."""
    import multiprocessing as mp
    import os
    saved = {k: os.environ.get(k) for k in _BLAS_VARS}
    for k in _BLAS_VARS:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(processes)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _eval_star(args):
    grid, genome, kw = args
    return evaluate(grid, genome, **kw)


def evaluate_many(grid, genomes, processes=1, **kw):
    """Evaluate several topologies, optionally across host processes (spawn)."""
    jobs = [(grid, g, kw) for g in genomes]
    if processes <= 1 or len(jobs) <= 1:
        return [_eval_star(j) for j in jobs]
    with _pool(processes) as pool:
        return pool.map(_eval_star, jobs, chunksize=1)


def _eval_chunk(args):
    grid, genome, chunk, kw = args
    return evaluate(grid, genome, outages=chunk, **kw)


def evaluate_parallel_outages(grid, genome, processes=8, **kw):
    """Brute-force evaluation of one topology with its outage re-solves spread
    over host processes (spawn); the per-process maxima are combined by max and
    the metrics recomputed from the combined f^max with the same formulas as
    :func:`evaluate`."""
    O = grid.outages.size
    chunks = [c for c in np.array_split(np.arange(O), max(1, processes)) if c.size]
    jobs = [(grid, genome, c, kw) for c in chunks]
    with _pool(len(jobs)) as pool:
        parts = pool.map(_eval_chunk, jobs, chunksize=1)
    r = dict(parts[0])
    if r["island_base"]:
        return r
    fmax = parts[0]["fmax"]
    for q in parts[1:]:
        fmax = np.maximum(fmax, q["fmax"])
    n_isl = sum(q["n_islanded"] for q in parts)
    lim = grid.limit[grid.monitored.astype(np.int64)]
    fprime = r["fprime"]
    lam_o = float(np.maximum(fmax - lim[None, :], 0.0).sum())
    lam_c = int((fmax > lim[None, :]).sum())
    lam_c0 = int((np.abs(fprime) > lim[None, :]).sum())
    maxload = float(np.max(np.maximum(np.abs(fprime), fmax) / lim[None, :]))
    r.update(fmax=fmax, n_islanded=n_isl, island_any=n_isl > 0, lambda_o=lam_o, lambda_c=lam_c,
             lambda_c0=lam_c0, maxload=maxload, fitness=-(lam_o + maxload),
             lambda_f1=-(lam_o + 200.0 * lam_c0 + 50.0 * lam_c))
    if kw.get("want_energy"):
        energy = np.full(O, np.nan)
        for q in parts:
            e = q["outage_energy"]
            energy[~np.isnan(e)] = e[~np.isnan(e)]
        r["outage_energy"] = energy
    return r
