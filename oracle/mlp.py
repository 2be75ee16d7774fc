"""FP64 surrogate network and its features (test oracle).

The surrogate screens mutated proposals before exact N-1 evaluation.  It is not
part of the paper; its definition here follows the workload description: an MLP
with three hidden layers of width H (ReLU), trained with mean squared error and
Adam (Kingma & Ba, 2015) to predict log1p(-fitness) of a topology, standardised
by the mean and deviation of the targets it has seen (``target_stats``).

Input (dimension 8 S + R): for every station s, eight values, non-zero only when
the genome splits s --
  [1, min(|A|,|B|)/m, b(B)/b(station), p_B / sum|p|, branches(B)/branches(station),
   |B|/m, 0, 0]
(m assets, |A|/|B| assets per busbar, b(.) summed susceptance of the branches,
p_B the injection on busbar B at timestep 0) -- followed by the post-split N-0
loading |f'_l| / fbar_l at timestep 0 of the R branches with the highest base-case
loading (descending, ties by branch id).

Parameters (layout shared with the library's description, not its code):
W1 [H][8S + R], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], w4 [H], b4 scalar.
"""
from __future__ import annotations

import numpy as np

from . import dcflow


def top_loaded_branches(grid, R):
    """The R branch ids of highest |f0(t=0)| / limit in the unsplit grid."""
    f0 = dcflow.base_flows(grid)[0]
    load = np.abs(f0) / grid.limit
    order = sorted(range(grid.n_branch), key=lambda l: (-load[l], l))
    return np.array(order[:R], dtype=np.int64)


def station_features(grid, genome):
    """Dense [S][8] station block of the input."""
    S = grid.n_station
    F = np.zeros((S, 8))
    psum = float(np.abs(grid.p[0]).sum())
    for a in genome:
        a = int(a)
        if a < 0:
            continue
        s = int(grid.action_station[a])
        mask = int(grid.action_mask[a])
        assets = grid.station_assets(s)
        m = len(assets)
        bus = int(grid.station_bus[s])
        onb = [(mask >> i) & 1 for i in range(m)]
        nb = sum(onb)
        br = [i for i in range(m) if assets[i] >= 0]
        b_all = sum(grid.b[assets[i]] for i in br)
        b_b = sum(grid.b[assets[i]] for i in br if onb[i])
        pb = sum(grid.p[0][bus] for i in range(m) if assets[i] < 0 and onb[i])
        F[s] = [1.0, min(nb, m - nb) / m, b_b / b_all, pb / psum,
                sum(1 for i in br if onb[i]) / len(br), nb / m, 0.0, 0.0]
    return F


def features(grid, genome, rows):
    """Full input vector (None when the split itself islands the grid)."""
    n_node, fr, to, p, _ = dcflow.post_split_graph(grid, genome)
    if not dcflow.is_connected_uf(n_node, fr, to):
        return None
    f = dcflow.solve_flows(n_node, fr, to, grid.b, p[:1], grid.slack)[0]
    xd = np.abs(f[rows]) / grid.limit[rows]
    return np.concatenate([station_features(grid, genome).ravel(), xd])


def init_params(D, H, seed=0):
    """He-uniform weights, zero biases (the same recipe the library uses; the
    tests copy one set of values into both)."""
    rng = np.random.default_rng(seed)

    def lin(n_out, n_in):
        lim = np.sqrt(6.0 / n_in)
        return rng.uniform(-lim, lim, (n_out, n_in))

    return dict(W1=lin(H, D), b1=np.zeros(H), W2=lin(H, H), b2=np.zeros(H), W3=lin(H, H),
                b3=np.zeros(H), w4=lin(1, H)[0], b4=np.zeros(1))


def forward(P, X):
    """Returns (y [M], cache)."""
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ P["w4"] + P["b4"][0]
    return y, (X, z1, h1, z2, h2, z3, h3)


def loss_and_grads(P, X, t):
    """L = mean((y - t)^2) and dL/dparams by the chain rule."""
    y, (X, z1, h1, z2, h2, z3, h3) = forward(P, X)
    M = X.shape[0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / M
    g = {}
    g["w4"] = h3.T @ dy
    g["b4"] = np.array([dy.sum()])
    d3 = np.outer(dy, P["w4"]) * (z3 > 0)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ P["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return L, g


def adam_step(P, G, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected first and second moments)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1 - beta1) * G[k]
        v[...] = beta2 * v + (1 - beta2) * G[k] * G[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P


def target(fitness):
    """log1p(-fitness) of a finite (non-positive) fitness."""
    return np.log1p(-np.asarray(fitness, dtype=np.float64))


def target_stats(t):
    """Mean and population standard deviation of the finite targets that the
    network's training targets are standardised with, (t - mean) / deviation:
    (0, 1) when there are none, deviation 1 when they are all equal."""
    t = np.asarray(t, dtype=np.float64)
    t = t[np.isfinite(t)]
    if t.size == 0:
        return 0.0, 1.0
    mean = float(np.sum(t) / t.size)
    sd = float(np.sqrt(np.sum((t - mean) ** 2) / t.size))
    return mean, (sd if sd > 0.0 else 1.0)
