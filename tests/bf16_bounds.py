"""Element-wise error bounds for one layer of the surrogate network computed
with BF16 operands and FP32 accumulation (test helper; no library code).

Error model (standard floating-point analysis, Higham, "Accuracy and Stability
of Numerical Algorithms", ch. 3): every product of the library's network rounds
its operands to BF16 (8 significant bits, unit roundoff U_BF16 = 2^-8) and sums
in FP32.  Tensor-core FP32 accumulation need not round to nearest, so each
accumulation step is charged V_ACC = 2^-22 (four times the FP32 unit roundoff).
For C = sum_k A_k B_k + bias over n terms, with A and B the layer's actual
inputs and operands rounded with unit roundoffs ua and ub:

  |C^ - C| <= c (|A| |B| + |bias|),  c = (1 + ua)(1 + ub)(1 + gamma_{n+1}) - 1,

with gamma_m = m V_ACC / (1 - m V_ACC).  A ReLU is 1-Lipschitz, and a ReLU mask
is taken from the library's own activations, so the bound carries over to the
masked and rectified values.

``check_layers`` applies this to every layer, forward and backward, with each
layer's inputs taken from the library's own trace (so errors do not compound
across layers the way a bound through the whole network would let them) and
returns, per quantity, the largest ratio of the error to its bound.  A
dropped term, a wrong sign or a transposed operand of ordinary size exceeds the
bound; ``emulate`` (the same arithmetic in numpy) lets the CPU tests show both
that the bounds hold and that such mistakes break them.
"""
from __future__ import annotations

import numpy as np

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24
V_ACC = 2.0 ** -22


def gamma(n, v=V_ACC):
    return n * v / (1.0 - n * v)


def coeff(n, ua=U_BF16, ub=U_BF16):
    return (1 + ua) * (1 + ub) * (1 + gamma(n + 1)) - 1


def _ratio(got, ref, bound):
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    bound = np.asarray(bound, dtype=np.float64)
    # an exact zero bound (an all-zero row) admits only an exact result
    return float(np.max(np.where(bound > 0, err / np.where(bound > 0, bound, 1.0),
                                 np.where(err > 0, np.inf, 0.0)))) if err.size else 0.0


def check_layers(P, X, tr, G=None, fit=None, station_cols=0):
    """Per-layer element-wise checks of a traced forward (and backward) pass.

    P: FP64 copies of the FP32 parameters (keys of oracle/mlp.py); X: the
    library's own inputs [M][D] (FP32 values); tr: trace dict with h [3][M][H]
    and y [M], and for a backward pass t, dy, dh [3][M][H]; G: the library's
    gradient blocks; fit: the FP32 fitness values the targets came from
    (targets unscaled: mean 0, deviation 1).  Returns {quantity: max err/bound}.
    """
    X = np.asarray(X, dtype=np.float64)
    h1, h2, h3 = (np.asarray(a, dtype=np.float64) for a in tr["h"])
    y = np.asarray(tr["y"], dtype=np.float64)
    W1, W2, W3, w4 = P["W1"], P["W2"], P["W3"], P["w4"]
    D, H = W1.shape[1], W2.shape[0]
    out = {}
    z = X @ W1.T + P["b1"]
    out["h1"] = _ratio(h1, np.maximum(z, 0), coeff(D) * (np.abs(X) @ np.abs(W1).T + np.abs(P["b1"])))
    z = h1 @ W2.T + P["b2"]
    out["h2"] = _ratio(h2, np.maximum(z, 0), coeff(H) * (h1 @ np.abs(W2).T + np.abs(P["b2"])))
    z = h2 @ W3.T + P["b3"]
    out["h3"] = _ratio(h3, np.maximum(z, 0), coeff(H) * (h2 @ np.abs(W3).T + np.abs(P["b3"])))
    out["y"] = _ratio(y, h3 @ w4 + P["b4"][0], coeff(H) * (h3 @ np.abs(w4) + abs(P["b4"][0])))
    if G is None:
        return out
    M = X.shape[0]
    t = np.asarray(tr["t"], dtype=np.float64)
    dy = np.asarray(tr["dy"], dtype=np.float64)
    d1, d2, d3 = (np.asarray(a, dtype=np.float64) for a in tr["dh"])
    t_ref = np.log1p(-np.asarray(fit, dtype=np.float64))
    out["t"] = _ratio(t, t_ref, 2 * U_FP32 * np.abs(t_ref))  # log1pf: 1 ulp
    r = y - t
    out["dy"] = _ratio(dy, 2.0 * r / M, 3 * U_FP32 * np.abs(2.0 * r / M))
    # output layer: w4 and b4 gradients are FP32 sums without BF16 rounding
    out["w4"] = _ratio(G["w4"], h3.T @ dy, coeff(M, 0, 0) * (h3.T @ np.abs(dy)))
    out["b4"] = _ratio(G["b4"], [dy.sum()], [gamma(M) * np.abs(dy).sum()])
    m3 = h3 > 0
    out["dh3"] = _ratio(d3, m3 * np.outer(dy, w4), coeff(1, 0) * m3 * np.abs(np.outer(dy, w4)))
    out["W3"] = _ratio(G["W3"], d3.T @ h2, coeff(M) * (np.abs(d3).T @ h2))
    out["b3"] = _ratio(G["b3"], d3.sum(axis=0), gamma(M) * np.abs(d3).sum(axis=0))
    m2 = h2 > 0
    out["dh2"] = _ratio(d2, m2 * (d3 @ W3), coeff(H) * m2 * (np.abs(d3) @ np.abs(W3)))
    out["W2"] = _ratio(G["W2"], d2.T @ h1, coeff(M) * (np.abs(d2).T @ h1))
    out["b2"] = _ratio(G["b2"], d2.sum(axis=0), gamma(M) * np.abs(d2).sum(axis=0))
    m1 = h1 > 0
    out["dh1"] = _ratio(d1, m1 * (d2 @ W2), coeff(H) * m1 * (np.abs(d2) @ np.abs(W2)))
    S8 = station_cols
    # station block: the backward signal is not rounded to BF16, the inputs are
    out["W1_station"] = _ratio(G["W1"][:, :S8], d1.T @ X[:, :S8],
                               coeff(M, 0) * (np.abs(d1).T @ np.abs(X[:, :S8])))
    out["W1_loads"] = _ratio(G["W1"][:, S8:], d1.T @ X[:, S8:], coeff(M) * (np.abs(d1).T @ np.abs(X[:, S8:])))
    out["b1"] = _ratio(G["b1"], d1.sum(axis=0), gamma(M) * np.abs(d1).sum(axis=0))
    return out


# ------------------------------------------------------------------ emulation
def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    i = a.view(np.uint32).astype(np.uint64)
    r = ((i + 0x7FFF + ((i >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def emulate(P, X, fit, station_cols):
    """The network's arithmetic as the error model describes it (BF16
    operands, FP32 sums), in numpy: a stand-in for the library with which the
    CPU tests show that the bounds hold and are not vacuous.  Returns (trace,
    gradient blocks)."""
    f = {k: np.asarray(v, dtype=np.float32) for k, v in P.items()}
    X = np.asarray(X, dtype=np.float32)
    S8 = station_cols
    h1 = np.maximum(bf16(X) @ bf16(f["W1"]).T + f["b1"], 0)
    h2 = np.maximum(bf16(h1) @ bf16(f["W2"]).T + f["b2"], 0)
    h3 = np.maximum(bf16(h2) @ bf16(f["W3"]).T + f["b3"], 0)
    y = bf16(h3) @ bf16(f["w4"]) + f["b4"][0]
    M = X.shape[0]
    t = np.log1p(-np.asarray(fit, dtype=np.float64)).astype(np.float32)
    dy = np.float32(2) * (y - t) / np.float32(M)
    G = {"w4": (h3 * dy[:, None]).sum(axis=0), "b4": np.array([dy.sum()], dtype=np.float32)}
    d3 = np.where(h3 > 0, dy[:, None] * bf16(f["w4"])[None, :], 0).astype(np.float32)
    G["W3"] = bf16(d3).T @ bf16(h2)
    G["b3"] = d3.sum(axis=0)
    d2 = np.where(h2 > 0, bf16(d3) @ bf16(f["W3"]), 0).astype(np.float32)
    G["W2"] = bf16(d2).T @ bf16(h1)
    G["b2"] = d2.sum(axis=0)
    d1 = np.where(h1 > 0, bf16(d2) @ bf16(f["W2"]), 0).astype(np.float32)
    W1 = np.empty_like(f["W1"])
    W1[:, :S8] = d1.T @ bf16(X[:, :S8])
    W1[:, S8:] = bf16(d1).T @ bf16(X[:, S8:])
    G["W1"] = W1
    G["b1"] = d1.sum(axis=0)
    tr = dict(h=np.stack([h1, h2, h3]), y=y, t=t, dy=dy, dh=np.stack([d1, d2, d3]))
    return tr, G
