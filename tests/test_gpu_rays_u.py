"""Per-ray mean intensity (mgx_solve_u) against the oracle, its consistency with
J (Eqs. 3-4), and the adaptive-vs-dense ray-set experiment of Section 3.2 on a
small wind: rays of the finest level are dense rays (error 0), and every other
adaptive ray is compared with the mean of the dense rays in its pixel.  Also the
reduction experiment of Table 2 on a small octree."""
import numpy as np
import pytest

from helpers import j_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    c = mgx.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("order", [2, 4])
def test_solve_u_parity_and_J(ctx, orc, order):
    import synth

    import paper_2011_14998_gb300 as mgx

    m = synth.random_cloud(150, seed=6, n_lines=2, n_freq=11, x_span=3.0, l_min=0, l_max=2, v_rms=1.0)
    mid = ctx.load(m)
    rays = ctx.rays(mid)
    o0, o1 = 17, 61
    u64 = ctx.solve_u(mid, o0, o1, precision=mgx.MGX_FP64, order=order, I_bdy=0.1)
    u32 = ctx.solve_u(mid, o0, o1, precision=mgx.MGX_FP32, order=order, I_bdy=0.1)
    J64 = ctx.solve_J(mid, precision=mgx.MGX_FP64, order=order, I_bdy=0.1)
    with pytest.raises(mgx.MgxError):
        ctx.solve_u(mid, 100, 151)
    ctx.free(mid)
    om = orc.OracleModel(m, rays=rays)
    o = np.arange(o0, o1)
    uo = om.solve_u(orc.params(order=order, I_bdy=0.1), o)
    assert u64.shape == uo.shape == (o1 - o0, rays.shape[1], 22)
    assert j_rel_err(u64.reshape(-1, 22), uo.reshape(-1, 22))[0] < 1e-10
    assert j_rel_err(u32.reshape(-1, 22), uo.reshape(-1, 22))[0] < 1e-4
    w2 = 2.0 / (12.0 * 4.0 ** (rays[o0:o1] >> 28))
    assert np.allclose((w2[:, :, None] * u64).sum(1), J64[o0:o1], rtol=1e-13, atol=0)


def test_adaptive_vs_dense_experiment(ctx):
    import synth

    from paper_2011_14998_gb300 import experiments

    m = synth.wind_model(2000, seed=9, n_freq=20)
    res = experiments.adaptive_vs_dense(ctx, m, origins=[3, 500, 1200, 1999], l_min=1, l_max=3)
    import paper_2011_14998_gb300 as mgx

    assert res["rays_adaptive"] == 2 * mgx.mgx_rayset_npairs(1, 3)
    assert res["rays_dense"] == 12 * 4**3
    assert 0 < res["frac_rays_at_finest_level"] < 1
    assert res["max_err_finest_level"] == 0.0  # the finest adaptive rays are dense rays
    assert 0.0 <= res["frac_rays_below_10pct"] <= res["frac_rays_below_20pct"] <= 1.0
    assert res["J_rel_err_mean"] < 0.2


def test_reduction_speedup_experiment(ctx):
    import synth

    from paper_2011_14998_gb300 import experiments

    m = synth.octree_model(8000, seed=12, hi_level=6, n_lines=1, n_freq=20, l_min=1, l_max=1)
    res = experiments.reduction_speedup(ctx, m, 0.90, 2.10, 0.10, reps=2)
    assert res["n_reduced"] < res["n_original"]
    assert res["speedup"] > 1.0
    assert np.isfinite(res["mean_rel_err"])


def test_reduction_sweep_speedup_grows(ctx):
    """Table 2 / Fig. 6 shape on the clump octree: stronger plain reductions give
    larger solve speed-ups, and the per-point error CDF is a distribution."""
    import synth

    from paper_2011_14998_gb300 import experiments

    m = synth.octree_model(20000, seed=12, hi_level=7, n_lines=1, n_freq=20, l_min=1, l_max=1)
    res = experiments.reduction_sweep(ctx, m, (0.90, 2.10, 0.10), scales=(1.0, 1.6, 2.6), reps=3)
    runs = res["runs"]
    red = [r["reduction"] for r in runs]
    spd = [r["speedup"] for r in runs]
    assert red[0] < red[1] < red[2]
    assert spd[0] < spd[1] < spd[2], spd
    for r in runs:
        c = np.asarray(r["cdf"])
        assert len(c) == 1000 and np.all(np.diff(c) >= 0) and abs(c[-1] - 1.0) < 1e-12
        assert np.isfinite(r["mean_rel_err"])
