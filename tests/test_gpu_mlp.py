"""BF16 tensor-core kernels of the learned reduction network against the FP64
NumPy oracle that rounds to bfloat16 at the same places: forward outputs,
per-layer gradients, training progress, input features and top-k selection.
Row counts are not multiples of the 64-point CTA tile (ragged tails)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    c = mgx.Context(0)
    yield c
    c.close()


def _layers(g):
    from oracle import mlp

    return mlp.unpack(g)


def test_forward_matches_oracle(ctx):
    import paper_2011_14998_gb300 as mgx
    from oracle import mlp

    theta = mlp.init(3)
    theta[mlp.NPARAM - 1] = 0.3
    X = np.random.default_rng(1).normal(size=(1001, 8)).astype(np.float32)
    mgx.mgx_mlp_set_params(ctx.ptr, theta)
    y = mgx.mgx_mlp_forward(ctx.ptr, X)
    yo, _ = mlp.forward(mgx.mgx_mlp_get_params(ctx.ptr).astype(np.float64), X, bf=True)
    assert np.all(np.abs(y - yo) <= 2e-3 * (np.abs(yo) + 1.0)), np.abs(y - yo).max()


def test_gradient_matches_oracle(ctx):
    import paper_2011_14998_gb300 as mgx
    from oracle import mlp

    rng = np.random.default_rng(2)
    theta = mlp.init(4)
    X = rng.normal(size=(777, 8)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.3 * X[:, 1] ** 2).astype(np.float32)
    mgx.mgx_mlp_set_params(ctx.ptr, theta)
    g, loss = mgx.mgx_mlp_grad(ctx.ptr, X, t)
    Lo, go = mlp.loss_and_grad(mgx.mgx_mlp_get_params(ctx.ptr).astype(np.float64), X, t, bf=True)
    assert loss == pytest.approx(Lo, rel=5e-3)
    # element by element: every gradient entry within 2^-6 (two bfloat16 units) of the sum of the
    # magnitudes of the terms it adds up; a transposed or shifted block fails this
    mag = mlp.grad_magnitudes(mgx.mgx_mlp_get_params(ctx.ptr).astype(np.float64), X, t, bf=True)
    gl, gol, ml = _layers(g), _layers(go), _layers(mag)
    for name in gl:
        bad = np.abs(gl[name] - gol[name]) > 2.0 ** -6 * ml[name] + 1e-9
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(gl[name] - gol[name]).max()))
    # the bound is tight enough to see a transposed W2 block
    W2 = gol["W2"]
    assert (np.abs(W2.T - W2) > 2.0 ** -6 * ml["W2"] + 1e-9).any()


def test_training_reduces_loss(ctx):
    import paper_2011_14998_gb300 as mgx
    from oracle import mlp

    rng = np.random.default_rng(5)
    X = rng.normal(size=(5000, 8)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * np.abs(X[:, 3])).astype(np.float32)
    mgx.mgx_mlp_set_params(ctx.ptr, mlp.init(6))
    losses = mgx.mgx_mlp_train(ctx.ptr, X, t, epochs=40, batch=256, lr=3e-3, seed=9)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0], losses
    # the trained parameters reproduce the reported loss through the oracle
    yo, _ = mlp.forward(mgx.mgx_mlp_get_params(ctx.ptr).astype(np.float64), X, bf=True)
    assert np.mean((yo - t) ** 2) < 0.3 * losses[0]


def test_features_match_oracle(ctx):
    import synth

    import paper_2011_14998_gb300 as mgx
    from oracle import mlp

    m = synth.wind_model(700, seed=41, n_freq=5)
    mid = ctx.load(m, rays=False)
    X = mgx.mgx_mlp_features(ctx.ptr, mid, m["rho"], m["T"])
    ctx.free(mid)
    Xo = mlp.features(m["pos"], m["vel"], m["nbr_off"], m["nbr_idx"], m["rho"], m["T"], m["dvw"], m["chi0"][:, 0])
    assert np.allclose(X, Xo, rtol=2e-5, atol=2e-5)


def test_learned_reduction_keeps_top_scores(ctx):
    import synth

    import paper_2011_14998_gb300 as mgx
    from oracle import mlp

    m = synth.wind_model(900, seed=42, n_freq=5)
    mid = ctx.load(m, rays=False)
    X = np.random.default_rng(7).normal(size=(900, 8)).astype(np.float32)
    mgx.mgx_mlp_set_params(ctx.ptr, mlp.init(8))
    y = mgx.mgx_mlp_forward(ctx.ptr, X)
    keep, k = mgx.mgx_reduce_mesh_learned(ctx.ptr, mid, X, 0.15)
    ctx.free(mid)
    assert k == round(0.15 * 900) and keep.sum() == k
    order = sorted(range(900), key=lambda i: (-float(y[i]), i))
    assert set(np.where(keep)[0]) == set(order[:k])
