"""Pins of the oracle MLP (learned reduction): its manual backward against
central finite differences of its forward, and structural special cases."""
import numpy as np
import pytest


def test_gradient_matches_finite_differences():
    from oracle import mlp

    rng = np.random.default_rng(0)
    theta = mlp.init(1) + rng.normal(0, 0.05, mlp.NPARAM)
    X = rng.normal(size=(40, 8))
    t = rng.normal(size=40)
    L, g = mlp.loss_and_grad(theta, X, t)
    idx = rng.choice(mlp.NPARAM, 120, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 8 * 64]])  # b3, W1[0,0], b1[0]
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAM)
        e[k] = h
        Lp, _ = mlp.loss_and_grad(theta + e, X, t)
        Lm, _ = mlp.loss_and_grad(theta - e, X, t)
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-8), k


def test_zero_hidden_weights_give_constant_output():
    from oracle import mlp

    p = mlp.unpack(np.zeros(mlp.NPARAM))
    p = {k: v.copy() for k, v in p.items()}
    p["b3"][0] = 0.7
    theta = mlp.pack(p)
    X = np.random.default_rng(2).normal(size=(10, 8))
    y, _ = mlp.forward(theta, X)
    assert np.allclose(y, 0.7)
    L, g = mlp.loss_and_grad(theta, X, np.zeros(10))
    gp = mlp.unpack(g)
    assert np.allclose(gp["W1"], 0) and np.allclose(gp["W2"], 0) and np.allclose(gp["W3"], 0)
    assert gp["b3"][0] == pytest.approx(2 * 0.7)


def test_bf16_rounding():
    from oracle import mlp

    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0  # tie to even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    x = np.random.default_rng(3).normal(size=1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2 ** -8)


def test_features_by_hand():
    """The eight features on a hand-built 4-point graph: a path 0-1-2 along x
    (unit spacing) plus an isolated point 3."""
    from oracle import mlp

    pos = np.array([[1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0], [0.0, 0, 5.0]])
    vel = np.array([[0.0, 0, 0], [3.0, 4.0, 0], [0.0, 0, 0], [1.0, 1, 1]])
    off = np.array([0, 1, 3, 4, 4])
    nbr = np.array([1, 0, 2, 1], np.int32)
    rho = np.array([1.0, np.e, np.e ** 3, 2.0])
    T = np.array([100.0, 200.0, 300.0, 400.0])
    dvw = np.array([0.5, 1.0, 2.0, 4.0])
    chi0 = np.array([2.0, 3.0, 4.0, 5.0])
    X = mlp.features(pos, vel, off, nbr, rho, T, dvw, chi0)
    # point 0: one neighbour (1) at distance 1, log rho contrast 1, |dv| = 5 over width 0.5
    assert X[0] == pytest.approx([0.0, 1.0, 10.0, np.log(100.0), 0.0, 1.0, 0.0, np.log(2.0)])
    # point 1: neighbours 0 and 2 at distance 1, contrasts 1 and 2, |dv| = 5 to both over width 1
    assert X[1] == pytest.approx([1.0, 2.0, 5.0, np.log(200.0), 0.0, 2.0, np.log(2.0), np.log(3.0)])
    # point 2: neighbour 1, contrast 2, |dv| = 5 over width 2
    assert X[2] == pytest.approx([3.0, 2.0, 2.5, np.log(300.0), 0.0, 1.0, np.log(3.0), np.log(4.0)])
    # point 3: no neighbours (mean distance 0, so log L and log(chi0 L) take the 1e-30 floor)
    assert X[3] == pytest.approx([np.log(2.0), 0.0, 0.0, np.log(400.0), np.log(1e-30), 0.0, np.log(5.0),
                                  np.log(1e-30)])
