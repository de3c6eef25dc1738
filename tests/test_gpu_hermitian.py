"""GPU parity of the Hermitian (fourth-order) scheme (Section 2.1, Auer 1976,
third-order boundary conditions) against the oracle's Hermitian solve: FP64
within 1e-10, FP32 within 1e-4 of the single-precision-decision oracle, through
the per-model, batched (graph replay) and allocation-free entry points.  The
cases include boundary origins (one empty half), an isolated point (both
empty), several lines and adaptive ray sets, and the 16^3 cube whose axis rays
have vanishing increments."""
import numpy as np
import pytest

from helpers import j_rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    c = mgx.Context(0)
    yield c
    c.close()


def _case(name):
    import synth

    if name == "grid16":
        return synth.grid_model(16), dict(dtau_max=0.2), np.arange(0, 4096, 5)
    if name == "wind":
        return synth.wind_model(1200, seed=23, n_freq=50, level=1), dict(), np.arange(0, 1200, 3)
    if name == "cloud":
        m = synth.random_cloud(120, seed=3, n_lines=3, n_freq=13, x_span=3.5, l_min=0, l_max=2, v_rms=1.5)
        return m, dict(dtau_max=0.3, I_bdy=0.2), np.arange(120)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["grid16", "wind", "cloud"])
def test_hermitian_fp64_and_fp32(ctx, orc, name):
    import paper_2011_14998_gb300 as mgx

    m, kw, origins = _case(name)
    mid = ctx.load(m)
    rays = ctx.rays(mid)
    J64 = ctx.solve_J(mid, precision=mgx.MGX_FP64, order=4, **kw)
    J32 = ctx.solve_J(mid, precision=mgx.MGX_FP32, order=4, **kw)
    J2 = ctx.solve_J(mid, precision=mgx.MGX_FP64, order=2, **kw)
    ctx.free(mid)
    om = orc.OracleModel(m, rays=rays)
    Jo = om.solve_J(orc.params(order=4, **kw), origins=origins)
    assert j_rel_err(J64[origins], Jo)[0] < FP64_TOL
    assert j_rel_err(J32[origins], Jo)[0] < FP32_TOL
    assert not np.array_equal(J64, J2)  # the order parameter reaches the kernel


def test_hermitian_boundary_and_isolated_points(ctx, orc):
    import synth

    import paper_2011_14998_gb300 as mgx

    m = synth.random_cloud(60, seed=11, n_freq=9, l_min=0, l_max=1)
    # an isolated point far outside the cloud: both halves of every pair are empty
    m["pos"] = np.vstack([m["pos"], [[5.0, 5.0, 5.0]]])
    for k in ("vel",):
        m[k] = np.vstack([m[k], [[0.0, 0.0, 0.0]]])
    for k in ("chi0", "eta0"):
        m[k] = np.vstack([m[k], m[k][:1]])
    for k in ("dvw", "chi_c", "eta_c", "rho", "T"):
        m[k] = np.concatenate([m[k], m[k][:1]])
    m["nbr_off"] = np.concatenate([m["nbr_off"], m["nbr_off"][-1:]])
    mid = ctx.load(m)
    rays = ctx.rays(mid)
    J64 = ctx.solve_J(mid, precision=mgx.MGX_FP64, order=4, I_bdy=0.3)
    ctx.free(mid)
    Jo = orc.OracleModel(m, rays=rays).solve_J(orc.params(order=4, I_bdy=0.3))
    assert np.allclose(J64[-1], 0.3, rtol=1e-14)  # u = I on every pair, weights sum to one
    assert j_rel_err(J64, Jo)[0] < FP64_TOL


def test_hermitian_batched_graph_and_noalloc(ctx, orc):
    import torch

    import synth

    import paper_2011_14998_gb300 as mgx

    models = [synth.wind_model(700, seed=41, n_freq=40, level=1),
              synth.octree_model(1500, seed=42, hi_level=5, n_lines=2, n_freq=20)]
    mids = [ctx.load(m) for m in models]
    singles32 = [ctx.solve_J(k, precision=mgx.MGX_FP32, order=4) for k in mids]
    flags = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS
    outs = ctx.solve_J_batch(mids, precision=mgx.MGX_FP32, flags=flags, order=4)
    ctx.solve_J_batch(mids, precision=mgx.MGX_FP32, outs=outs, flags=flags, order=4)  # replay
    for o, s in zip(outs, singles32):
        assert j_rel_err(o.cpu().numpy(), s)[0] < 1e-5
    J64 = ctx.solve_J(mids[0], precision=mgx.MGX_FP64, order=4)
    out = torch.empty(J64.shape, dtype=torch.float64, device="cuda")
    mgx.mgx_solve_J_noalloc(ctx.ptr, mids[0], mgx.solve_params(precision=mgx.MGX_FP64, order=4), out)
    assert np.array_equal(out.cpu().numpy(), J64)
    rays = ctx.rays(mids[1])
    for k in mids:
        ctx.free(k)
    om = orc.OracleModel(models[1], rays=rays)
    o = np.arange(0, len(models[1]["pos"]), 11)
    Jo = om.solve_J(orc.params(order=4), origins=o)
    assert j_rel_err(outs[1].cpu().numpy()[o], Jo)[0] < FP32_TOL


def test_invalid_order_rejected(ctx):
    import synth

    import paper_2011_14998_gb300 as mgx

    mid = ctx.load(synth.grid_model(4, n_freq=3))
    with pytest.raises(mgx.MgxError):
        ctx.solve_J(mid, order=3)
    ctx.free(mid)
