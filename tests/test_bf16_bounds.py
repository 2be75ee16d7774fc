"""The per-layer BF16 error bounds used by the surrogate's GPU parity tests
hold for an emulation of BF16-operand / FP32-sum arithmetic and are not
vacuous: a dropped term, a sign error or a transposed operand in one layer of
the emulated network exceeds them."""
import numpy as np
import pytest

from oracle import mlp
from tests import bf16_bounds as bb


def _case(seed, M=96, H=64, S=10, R=40):
    rng = np.random.default_rng(seed)
    D = 8 * S + R
    P = mlp.init_params(D, H, seed=seed)
    for k in ["b1", "b2", "b3", "b4"]:
        P[k] = rng.normal(0, 0.05, P[k].shape)
    P = {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}
    X = np.zeros((M, D))
    for m in range(M):  # up to 3 split stations per row, 6 non-zero values each
        for s in rng.choice(S, rng.integers(1, 4), replace=False):
            X[m, 8 * s: 8 * s + 6] = np.r_[1.0, rng.random(5)]
    X[:, 8 * S:] = rng.uniform(0.0, 1.5, (M, R))
    X = X.astype(np.float32).astype(np.float64)
    y, _ = mlp.forward(P, X)
    fit = (-np.expm1(y + rng.uniform(1.0, 2.0, M))).astype(np.float32)
    return P, X, fit, 8 * S


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_emulated_layers_within_bounds(seed):
    P, X, fit, S8 = _case(seed)
    tr, G = bb.emulate(P, X, fit, S8)
    r = bb.check_layers(P, X, tr, G, fit, S8)
    assert max(r.values()) <= 1.0, r
    # not vacuous: the products' rounding uses a visible share of the bound
    for k in ["h1", "h2", "h3", "y", "dh2", "dh1", "W3", "W2", "W1_loads"]:
        assert r[k] > 0.01, (k, r[k])


def _break(P, X, fit, S8, what):
    """Emulated pass with one planted mistake."""
    tr, G = bb.emulate(P, X, fit, S8)
    tr = {k: np.array(v, dtype=np.float32) for k, v in tr.items()}
    G = {k: np.array(v, dtype=np.float32) for k, v in G.items()}
    if what == "dropped W2 column":
        P2 = dict(P)
        W2 = P["W2"].copy()
        W2[:, 7] = 0.0
        P2["W2"] = W2
        tr2, _ = bb.emulate(P2, X, fit, S8)
        tr["h"][1] = tr2["h"][1]
    elif what == "transposed W3":
        P2 = dict(P)
        P2["W3"] = P["W3"].T.copy()
        tr2, _ = bb.emulate(P2, X, fit, S8)
        tr["h"][2] = tr2["h"][2]
    elif what == "dropped station slice":
        Xs = X.copy()
        row = int(np.flatnonzero(X[:, :S8].any(axis=1))[0])
        col = int(np.flatnonzero(X[row, :S8])[0])
        Xs[row, col: col + 6] = 0.0
        tr2, _ = bb.emulate(P, Xs, fit, S8)
        tr["h"][0][row] = tr2["h"][0][row]
    elif what.startswith("sign "):
        k = what.split()[1]
        if k in G:
            g = G[k].ravel()
            i = int(np.argsort(np.abs(g))[g.size // 2])  # an entry of median size
            g[i] = -g[i]
        else:
            d = tr["dh"][int(k[-1]) - 1].ravel()
            nz = np.flatnonzero(d)
            i = nz[np.argsort(np.abs(d[nz]))[nz.size // 2]]
            d[i] = -d[i]
    elif what == "transposed backward W2":
        d2 = tr["dh"][1]
        m1 = tr["h"][0] > 0
        tr["dh"][0] = np.where(m1, bb.bf16(d2) @ bb.bf16(P["W2"].T.astype(np.float32)), 0)
    return tr, G


@pytest.mark.parametrize("what", ["dropped W2 column", "transposed W3", "dropped station slice",
                                  "sign W3", "sign W2", "sign W1", "sign b1", "sign w4", "sign dh2",
                                  "sign dh1", "transposed backward W2"])
def test_planted_mistakes_exceed_bounds(what):
    P, X, fit, S8 = _case(7)
    tr, G = _break(P, X, fit, S8, what)
    r = bb.check_layers(P, X, tr, G, fit, S8)
    assert max(r.values()) > 1.0, (what, r)
