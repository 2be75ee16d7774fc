"""MapElites operators restated in plain Python (test oracle).

* Mutation: the action (split) part of Algorithm 1.  N_mut is drawn from a
  Poisson distribution with mean N_mutmean, clipped to [1, N_a]; each of the
  N_mut rounds draws one feasible operation among Add / Remove / Change /
  Identity with probabilities 0.2 / 0.2 / 0.5 / 0.1 (Sec. "Mutation
  Operation"), renormalised over the operations that are feasible for the
  current genome.  Add fills a random empty slot with an action of a station
  not yet in the genome; Remove clears a random filled slot; Change replaces
  the action of a random filled slot by a different action of the same station
  (the exclusion set s(a)).  A genome left without any split is forced through
  Add (the forced-change rule, applied to split slots because this genome has
  no disconnection slots).
* Parent selection: uniform over the filled archive cells, in ascending cell
  order (the paper does not state it); an empty archive yields the unsplit
  topology as parent (Algorithm 3 initialises the repertoire with it).
* Archive insert: Algorithm 3's sorted insert, read as one elite per cell and a
  candidate replacing it only when strictly better, candidates taken in batch
  order.

Every random decision compares a Philox word with an integer threshold
computed in FP64 from the probabilities, so an implementation that uses the
same thresholds and the same word order reproduces the draws bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import WordStream, uniform_index

ADD, REMOVE, CHANGE, IDENTITY = 0, 1, 2, 3
DEFAULT_PROBS = (0.2, 0.2, 0.5, 0.1)  # add, remove, change, identity
TWO32 = 4294967296.0


def op_thresholds(probs, feasible):
    """Cumulative uint32 thresholds over the feasible operations; the last
    feasible operation's threshold is 2^32 so that every word selects one."""
    w = [probs[i] if (feasible >> i) & 1 else 0.0 for i in range(4)]
    cum = []
    acc = 0.0
    for x in w:
        acc = acc + x
        cum.append(acc)
    total = cum[3]
    last = max(i for i in range(4) if w[i] > 0)
    thr = []
    for i in range(4):
        if i >= last:
            thr.append(1 << 32)
        else:
            thr.append(int(math.floor(cum[i] / total * TWO32)))
    return thr


def poisson_thresholds(mean, k_max):
    """uint32 thresholds floor(CDF(j) * 2^32), j = 0 .. k_max - 1, of a
    Poisson(mean) variable; the pmf follows p_0 = e^-mean, p_j = p_{j-1} mean / j."""
    pmf = math.exp(-mean)
    cdf = pmf
    thr = [int(math.floor(cdf * TWO32))]
    for j in range(1, k_max):
        pmf = pmf * mean / j
        cdf = cdf + pmf
        thr.append(int(math.floor(cdf * TWO32)))
    return thr


def draw_n_mut(word, pthr, k_max):
    n = k_max
    for j, t in enumerate(pthr):
        if word < t:
            n = j
            break
    return min(max(n, 1), k_max)


class ActionTable:
    def __init__(self, grid):
        self.off = np.asarray(grid.action_offset, dtype=np.int64)
        self.station = np.asarray(grid.action_station, dtype=np.int64)
        self.n_action = int(self.station.size)

    def count(self, s):
        return int(self.off[s + 1] - self.off[s])

    def sample_allowed(self, genome, word):
        """Uniform action among stations absent from the genome."""
        excl = sorted({int(self.station[a]) for a in genome if a >= 0})
        allowed = self.n_action - sum(self.count(s) for s in excl)
        pos = uniform_index(word, allowed)
        for s in excl:  # ascending action offsets
            if pos >= self.off[s]:
                pos += self.count(s)
            else:
                break
        return int(pos)


def feasibility(genome, tab):
    filled = [i for i, a in enumerate(genome) if a >= 0]
    empty = [i for i, a in enumerate(genome) if a < 0]
    excl = {int(tab.station[genome[i]]) for i in filled}
    allowed = tab.n_action - sum(tab.count(s) for s in excl)
    changeable = [i for i in filled if tab.count(int(tab.station[genome[i]])) >= 2]
    f = 0
    if empty and allowed > 0:
        f |= 1 << ADD
    if filled:
        f |= 1 << REMOVE
    if changeable:
        f |= 1 << CHANGE
    f |= 1 << IDENTITY
    return f, filled, empty, changeable


def _add(g, tab, ws):
    empty = [i for i, a in enumerate(g) if a < 0]
    slot = empty[uniform_index(ws.next(), len(empty))]
    g[slot] = tab.sample_allowed(g, ws.next())


def mutate(parent, tab, ws, probs=DEFAULT_PROBS, mean=2.0):
    """Algorithm 1 (action part) on one genome, consuming words from ``ws``
    (the parent-selection word has already been consumed)."""
    g = [int(a) for a in parent]
    k = len(g)
    pthr = poisson_thresholds(mean, k)
    n_mut = draw_n_mut(ws.next(), pthr, k)
    for _ in range(n_mut):
        feas, filled, empty, changeable = feasibility(g, tab)
        thr = op_thresholds(probs, feas)
        w = ws.next()
        op = next(i for i in range(4) if w < thr[i])
        if op == ADD:
            _add(g, tab, ws)
        elif op == REMOVE:
            slot = filled[uniform_index(ws.next(), len(filled))]
            g[slot] = -1
        elif op == CHANGE:
            slot = changeable[uniform_index(ws.next(), len(changeable))]
            s = int(tab.station[g[slot]])
            cur = g[slot] - int(tab.off[s])
            r = uniform_index(ws.next(), tab.count(s) - 1)
            g[slot] = int(tab.off[s]) + r + (1 if r >= cur else 0)
    if all(a < 0 for a in g):
        _add(g, tab, ws)
    return np.array(g, dtype=np.int32)


def propose(archive, tab, seed, iteration, B, k_max, probs=DEFAULT_PROBS, mean=2.0):
    """B mutated genomes from parents drawn uniformly over filled cells (the
    parent word is drawn even when the archive is empty)."""
    filled = sorted(archive.elites)
    out = []
    for cand in range(B):
        ws = WordStream(seed, iteration, cand)
        w = ws.next()
        if filled:
            parent = archive.elites[filled[uniform_index(w, len(filled))]][1]
        else:  # empty archive: mutate the pre-optimisation (unsplit) topology
            parent = np.full(k_max, -1, dtype=np.int32)
        out.append(mutate(parent, tab, ws, probs, mean))
    return np.stack(out)


class Archive:
    """One elite per cell: cell -> (fitness, genome)."""

    def __init__(self, d_split, d_moved):
        self.d_split = d_split
        self.d_moved = d_moved
        self.elites = {}

    def insert(self, cells, fitness, genomes):
        """Sequential insert in batch order with strict improvement; invalid
        (non-finite) fitness is never inserted.  Returns the number of cells
        changed."""
        changed = 0
        for c, f, g in zip(cells, fitness, genomes):
            if not np.isfinite(f):
                continue
            c = int(c)
            cur = self.elites.get(c)
            if cur is None or f > cur[0]:
                self.elites[c] = (float(f), np.array(g, dtype=np.int32))
                changed += 1
        return changed

    def best(self):
        return max(v[0] for v in self.elites.values())
