"""Batched, length-binned persistent solve (mgx_solve_J_batch) and its CUDA-graph
replay: same J as the per-model solve and as the oracle, for models of different
sizes, line counts, bin counts and ray sets in one launch."""
import numpy as np
import pytest

from helpers import j_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import synth

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    ctx = mgx.Context(0)
    models = [
        synth.wind_model(900, seed=31, n_freq=50, level=2),
        synth.random_cloud(150, seed=5, n_lines=3, n_freq=13, x_span=3.5, l_min=0, l_max=2, v_rms=1.5),
        synth.grid_model(6, n_freq=9),
        synth.wind_model(600, seed=32, n_freq=20, level=1, l_min=0),
    ]
    mids = [ctx.load(m) for m in models]
    yield ctx, models, mids
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (0, 1e-13)])
def test_batch_matches_single_model_solves(setup, prec, tol):
    ctx, models, mids = setup
    singles = [ctx.solve_J(m, precision=prec) for m in mids]
    outs = ctx.solve_J_batch(mids, precision=prec)
    for J1, Jb in zip(singles, outs):
        assert Jb.shape == J1.shape
        assert j_rel_err(Jb.cpu().numpy(), J1)[0] <= tol


def test_batch_against_oracle(setup, orc):
    ctx, models, mids = setup
    outs = ctx.solve_J_batch(mids, precision=0, dtau_max=0.4, I_bdy=0.05)
    for m, mid, Jb in zip(models, mids, outs):
        om = orc.OracleModel(m, rays=ctx.rays(mid))
        origins = np.arange(0, len(m["pos"]), 7)
        Jo = om.solve_J(orc.params(dtau_max=0.4, I_bdy=0.05), origins=origins)
        assert j_rel_err(Jb.cpu().numpy()[origins], Jo)[0] < 1e-10


def test_graph_replay_with_ray_rebuild(setup):
    import paper_2011_14998_gb300 as mgx

    ctx, models, mids = setup
    ref = ctx.solve_J_batch(mids, precision=1)
    outs = ctx.solve_J_batch(mids, precision=1, flags=mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS)
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    ctx.solve_J_batch(mids, precision=1, outs=outs, flags=mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS)  # replay
    for a, b, r in zip(first, outs, ref):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
        assert np.array_equal(a.cpu().numpy(), r.cpu().numpy())


def test_batch_rejects_bad_arguments(setup):
    import torch

    import paper_2011_14998_gb300 as mgx

    ctx, models, mids = setup
    out = torch.empty((900, 50), dtype=torch.float64, device="cuda")
    with pytest.raises(mgx.MgxError):  # a model twice
        mgx.mgx_solve_J_batch(ctx.ptr, [mids[0], mids[0]], mgx.solve_params(), [out, out])


def test_batch_host_outputs(setup):
    """Outputs in host memory (pageable and pinned, mixed with device memory)
    receive the same J as device outputs, in the eager step and in graph replays."""
    import torch

    import paper_2011_14998_gb300 as mgx

    ctx, models, mids = setup
    ref = [o.cpu().numpy() for o in ctx.solve_J_batch(mids, precision=1)]
    outs = []
    for k, o in enumerate(ref):
        if k % 3 == 0:
            outs.append(torch.full(o.shape, -1.0, dtype=torch.float64))
        elif k % 3 == 1:
            outs.append(torch.full(o.shape, -1.0, dtype=torch.float64).pin_memory())
        else:
            outs.append(torch.full(o.shape, -1.0, dtype=torch.float64, device="cuda"))
    params = mgx.solve_params(precision=mgx.MGX_FP32)
    for flags in (0, mgx.MGX_BATCH_GRAPH, mgx.MGX_BATCH_GRAPH):  # eager, plan + capture, replay
        for o in outs:
            o.fill_(-1.0)
        mgx.mgx_solve_J_batch(ctx.ptr, mids, params, outs, flags)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)


def test_tuning_changes_speed_not_results(setup):
    """The tracer grid, the row width and the work-list order never change J; the bins per lane
    select a differently compiled kernel, so single-precision J may differ in
    its rounding (fused multiply-adds), far inside the FP32 tolerance."""
    import paper_2011_14998_gb300 as mgx

    ctx, models, mids = setup
    flags = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS
    ctx.set_tuning(None)
    ref = [o.cpu().numpy() for o in ctx.solve_J_batch(mids, precision=1, flags=flags)]
    for t in ({"bins_per_lane": 2, "trace_ctas_per_sm": 4, "tail_permille": 5, "schedule": 0},
              {"bins_per_lane": 2, "trace_ctas_per_sm": 16, "tail_permille": 1000, "schedule": 1},
              {"bins_per_lane": 1, "trace_ctas_per_sm": 8, "tail_permille": 80, "schedule": 0}):
        ctx.set_tuning(t)
        assert ctx.tuning() == t
        outs = ctx.solve_J_batch(mids, precision=1, flags=flags)
        for o, r in zip(outs, ref):
            if t["bins_per_lane"] == 2:  # the automatic choice for this batch (up to 50 bins)
                assert np.array_equal(o.cpu().numpy(), r)
            else:
                assert j_rel_err(o.cpu().numpy(), r)[0] < 1e-5
    ctx.set_tuning(None)
    assert ctx.tuning() == {"bins_per_lane": 0, "trace_ctas_per_sm": 0, "tail_permille": 0, "schedule": 0}
    with pytest.raises(mgx.MgxError):
        ctx.set_tuning({"bins_per_lane": 3})
    with pytest.raises(mgx.MgxError):
        ctx.set_tuning({"trace_ctas_per_sm": 33})


def test_autotune_keeps_fastest_candidate(setup):
    import paper_2011_14998_gb300 as mgx

    ctx, models, mids = setup
    flags = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS
    ctx.set_tuning(None)
    ref = [o.cpu().numpy() for o in ctx.solve_J_batch(mids, precision=1, flags=flags)]
    trials, outs = ctx.autotune(mids, precision=1, flags=flags, reps=2)
    assert 5 <= len(trials) <= 10
    assert all(t["step_ms"] > 0 for t in trials)
    best = min(trials, key=lambda t: t["step_ms"])
    chosen = ctx.tuning()
    assert chosen == {k: best[k] for k in chosen}
    for o, r in zip(outs, ref):
        assert j_rel_err(o.cpu().numpy(), r)[0] < 1e-5
    ctx.set_tuning(None)
