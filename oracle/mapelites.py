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
* Disconnection mutation (the second part of Algorithm 1), for genomes with
  disconnection slots: after the split rounds one operation among Add /
  Remove / Change / Identity with probabilities 0.25 / 0.25 / 0.5 / 0 (same
  section), renormalised over the feasible ones (Identity when none has
  weight).  Add fills a random empty slot with a disconnection not in the
  genome (exclusion set phi = d); Remove clears a random filled slot; Change
  first draws a disconnection not in the genome, then the filled slot it
  replaces, in the order the algorithm lists.  A genome with neither a split
  nor a disconnection takes Add (the forced-change rule); the split forced Add
  then does not apply.
* Crossover (Algorithm 2): each child slot in turn takes an entry of the
  parents' union not yet in the child and feasible for it (distinct stations,
  distinct branches): with both parents offering one, parent 1's with
  probability p_c1; with one parent offering, that parent's if its weight
  (p_c1, or 1 - p_c1) is not zero; then uniformly among the chosen parent's
  remaining entries in slot order.  An entry both parents hold counts as
  parent 1's.  The first slot with nothing to take ends the part (the rest stay
  empty).  Algorithm 3 splits each batch: b_mc ~ Uniform{0, .., B} children
  by mutation, the rest by crossover of two parents drawn independently and
  uniformly over the filled cells.
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
DEFAULT_DPROBS = (0.25, 0.25, 0.5, 0.0)  # disconnection add, remove, change, identity
TWO32 = 4294967296.0
RATIO_STREAM = 0xFFFFFFFF  # candidate index of the per-iteration mutation/crossover draw


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


def dop_thresholds(probs, feasible):
    """As op_thresholds, but Identity when no feasible operation has weight."""
    if not any(probs[i] > 0 and (feasible >> i) & 1 for i in range(4)):
        return [0, 0, 0, 1 << 32]
    return op_thresholds(probs, feasible)


def p_c1_threshold(p_c1):
    """uint32 threshold of the parent-1 choice: floor(p_c1 2^32), 2^32 at 1."""
    return 1 << 32 if p_c1 >= 1.0 else int(math.floor(p_c1 * TWO32))


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


def _sample_free(d, n_disc, word):
    """Uniform disconnection index among those not in ``d``."""
    excl = sorted(int(x) for x in d if x >= 0)
    pos = uniform_index(word, n_disc - len(excl))
    for x in excl:
        if pos >= x:
            pos += 1
        else:
            break
    return pos


def mutate_disc(g, d, n_disc, ws, dprobs=DEFAULT_DPROBS):
    """The disconnection part of Algorithm 1 on the split slots ``g`` (already
    mutated) and the disconnection slots ``d`` (modified in place)."""
    filled = [i for i, x in enumerate(d) if x >= 0]
    empty = [i for i, x in enumerate(d) if x < 0]
    free = n_disc - len(filled)
    feas = 1 << IDENTITY
    if empty and free > 0:
        feas |= 1 << ADD
    if filled:
        feas |= 1 << REMOVE
    if filled and free > 0:
        feas |= 1 << CHANGE
    thr = dop_thresholds(dprobs, feas)
    w = ws.next()
    op = next(i for i in range(4) if w < thr[i])
    if not filled and all(a < 0 for a in g) and (feas >> ADD) & 1:
        op = ADD  # neither a split nor a disconnection: force one
    if op == ADD:
        slot = empty[uniform_index(ws.next(), len(empty))]
        d[slot] = _sample_free(d, n_disc, ws.next())
    elif op == REMOVE:
        d[filled[uniform_index(ws.next(), len(filled))]] = -1
    elif op == CHANGE:
        x = _sample_free(d, n_disc, ws.next())
        d[filled[uniform_index(ws.next(), len(filled))]] = x


def mutate(parent, tab, ws, probs=DEFAULT_PROBS, mean=2.0, n_dslot=0, n_disc=0, dprobs=DEFAULT_DPROBS):
    """Algorithm 1 on one genome (``n_dslot`` disconnection slots after the
    split slots), consuming words from ``ws`` (the parent-selection word has
    already been consumed)."""
    parent = [int(a) for a in parent]
    k_all = len(parent)
    g = parent[: k_all - n_dslot]
    d = parent[k_all - n_dslot:]
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
    if n_dslot > 0 and n_disc > 0:
        mutate_disc(g, d, n_disc, ws, dprobs)
    elif all(a < 0 for a in g):
        _add(g, tab, ws)
    return np.array(g + d, dtype=np.int32)


def _cross_part(x1, x2, width, key, ws, t_c1):
    child = []
    for _ in range(width):
        taken = {key(c) for c in child}
        s1 = {int(x) for x in x1 if x >= 0}
        r1 = [int(x) for x in x1 if x >= 0 and key(int(x)) not in taken]
        r2 = [int(x) for x in x2 if x >= 0 and int(x) not in s1 and key(int(x)) not in taken]
        if not r1 and not r2:
            break
        w = ws.next()
        if r1 and r2:
            from1 = w < t_c1
        elif r1:
            if t_c1 == 0:
                break
            from1 = True
        else:
            if t_c1 >= 1 << 32:
                break
            from1 = False
        r = r1 if from1 else r2
        child.append(r[uniform_index(ws.next(), len(r))])
    return child + [-1] * (width - len(child))


def crossover(p1, p2, tab, ws, n_dslot=0, p_c1=0.5):
    """Algorithm 2 on two parent genomes, consuming words from ``ws`` (the two
    parent-selection words have already been consumed)."""
    t_c1 = p_c1_threshold(p_c1)
    k = len(p1) - n_dslot
    a = _cross_part(p1[:k], p2[:k], k, lambda x: int(tab.station[x]), ws, t_c1)
    d = _cross_part(p1[k:], p2[k:], n_dslot, lambda x: x, ws, t_c1) if n_dslot else []
    return np.array(a + d, dtype=np.int32)


def mutation_count(seed, iteration, B, crossover_on):
    """b_mc of Algorithm 3: the children of one batch made by mutation."""
    if not crossover_on:
        return B
    return uniform_index(WordStream(seed, iteration, RATIO_STREAM).next(), B + 1)


def propose(archive, tab, seed, iteration, B, k_max, probs=DEFAULT_PROBS, mean=2.0, n_dslot=0, n_disc=0,
            dprobs=DEFAULT_DPROBS, crossover_on=False, p_c1=0.5):
    """B genomes from parents drawn uniformly over filled cells (each parent
    word is drawn even when the archive is empty, whose parent is the
    pre-optimisation topology): the first b_mc by mutation, the rest by
    crossover."""
    filled = sorted(archive.elites)
    empty = np.full(k_max + n_dslot, -1, dtype=np.int32)

    def pick(w):
        return archive.elites[filled[uniform_index(w, len(filled))]][1] if filled else empty

    b_mc = mutation_count(seed, iteration, B, crossover_on)
    out = []
    for cand in range(B):
        ws = WordStream(seed, iteration, cand)
        if cand < b_mc:
            parent = pick(ws.next())
            out.append(mutate(parent, tab, ws, probs, mean, n_dslot, n_disc, dprobs))
        else:
            p1 = pick(ws.next())
            p2 = pick(ws.next())
            out.append(crossover(p1, p2, tab, ws, n_dslot, p_c1))
    return np.stack(out)


class Archive:
    """One elite per cell: cell -> (fitness, genome)."""

    def __init__(self, d_split, d_moved, d_disc=1):
        self.d_split = d_split
        self.d_moved = d_moved
        self.d_disc = d_disc
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
