"""Pins of the FP64 surrogate oracle: gradients against central finite
differences, Adam against its closed form on a scalar quadratic, a trained
network reducing the loss, and the feature definitions on the 3-bus grid."""
import numpy as np
import pytest

from oracle import mlp
from tests.gridcases import three_bus, action_of


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    D, H, M = 11, 7, 5
    P = mlp.init_params(D, H, seed=1)
    for k in ["b1", "b2", "b3"]:
        P[k] = rng.normal(0, 0.1, P[k].shape)  # keep units active on both sides of zero
    X = rng.normal(size=(M, D))
    t = rng.normal(size=M)
    L, G = mlp.loss_and_grads(P, X, t)
    h = 1e-6
    for k in P:
        flat = P[k].ravel()
        for i in rng.choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[i]
            flat[i] = old + h
            Lp, _ = mlp.loss_and_grads(P, X, t)
            flat[i] = old - h
            Lm, _ = mlp.loss_and_grads(P, X, t)
            flat[i] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(G[k].ravel()[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, i)


def test_adam_closed_form_first_steps():
    # f(x) = x^2 / 2: gradient x.  Step 1 of Adam moves by lr * sign(g) (bias
    # correction makes m_hat = g and v_hat = g^2 exactly).
    P = {"x": np.array([3.0])}
    st = {}
    mlp.adam_step(P, {"x": P["x"].copy()}, st, lr=0.1)
    assert P["x"][0] == pytest.approx(3.0 - 0.1 * 3.0 / (3.0 + 1e-8), rel=1e-12)
    # step 2 with gradient g2: m = 0.9*0.1*g1 + 0.1*g2 ... written out by hand
    g1, g2 = 3.0, P["x"][0]
    mlp.adam_step(P, {"x": np.array([g2])}, st, lr=0.1)
    m = 0.9 * (0.1 * g1) + 0.1 * g2
    v = 0.999 * (0.001 * g1 * g1) + 0.001 * g2 * g2
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    assert P["x"][0] == pytest.approx(g2 - 0.1 * mh / (np.sqrt(vh) + 1e-8), rel=1e-12)


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    D, H, M = 6, 16, 64
    P = mlp.init_params(D, H, seed=3)
    X = rng.normal(size=(M, D))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2
    st = {}
    L0, _ = mlp.loss_and_grads(P, X, t)
    for _ in range(300):
        L, G = mlp.loss_and_grads(P, X, t)
        mlp.adam_step(P, G, st, lr=3e-3)
    assert L < 0.2 * L0


def test_station_features_three_bus():
    g, d = three_bus()
    # station at bus 1 with assets [branch 0 (0->1), branch 1 (1->2), injection]
    a = action_of(g, 0, 6)  # busbar B = {branch 1, injection}
    F = mlp.station_features(g, [a])
    psum = np.abs(g.p[0]).sum()
    np.testing.assert_allclose(F[0], [1.0, 1 / 3, 0.5, 1.0 / psum, 0.5, 2 / 3, 0.0, 0.0])
    x = mlp.features(g, [a], np.array([0, 1]))
    # post-split flows (0, 1, 0) against limits (0.5, 0.9)
    np.testing.assert_allclose(x[8:], [0.0, 1.0 / 0.9], atol=1e-12)


def test_target_stats_closed_forms():
    assert mlp.target_stats([1.0, 3.0]) == (2.0, 1.0)
    assert mlp.target_stats([1.0, np.nan, 3.0, np.inf, -np.inf]) == (2.0, 1.0)
    assert mlp.target_stats([5.0, 5.0, 5.0]) == (5.0, 1.0)
    assert mlp.target_stats([]) == (0.0, 1.0)
    m, sd = mlp.target_stats([0.0, 0.0, 0.0, 4.0])  # mean 1, squares 1+1+1+9 over 4
    assert m == 1.0 and sd == pytest.approx(np.sqrt(3.0), rel=1e-15)
    assert mlp.target([0.0, -np.e + 1.0]) == pytest.approx([0.0, 1.0], rel=1e-15)
