"""The single-precision form takes the integer decisions of the definition
(the velocity-sample count of Section 2.1.1 and Eq. 2's n_inter): each is
certified from a bound on the single-precision values' distance from the
double-precision ones, or redone in double precision.  These tests check the
bounds the certification rests on, and that the decisions agree with the FP64
oracle where single precision alone would land on another integer."""
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


def test_approximation_error_bounds(ctx):
    """ex2.approx over the exponents the profile uses (2^-a'^2 with a normal
    result) and rcp.approx over every mantissa pattern of several binades stay
    within half the relative error bounds the certification takes."""
    import torch

    import paper_2011_14998_gb300 as mgx

    rng = np.random.default_rng(1)
    x = np.concatenate([np.linspace(-126.0, 0.0, 1 << 22), -rng.uniform(0, 126, 1 << 20),
                        -np.arange(0, 127, dtype=np.float64)]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    b_ex2 = mgx.mgx_eval_approx(ctx.ptr, 0, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    ref = np.exp2(x.astype(np.float64))
    e_ex2 = float(np.max(np.abs(y - ref) / ref))
    mant = np.arange(1 << 23, dtype=np.uint32)
    r = np.concatenate([((127 + e) << 23 | mant).view(np.float32) for e in (-20, -1, 0, 1, 13)])
    rd = torch.from_numpy(r).cuda()
    qd = torch.empty_like(rd)
    b_rcp = mgx.mgx_eval_approx(ctx.ptr, 1, rd, qd)
    torch.cuda.synchronize()
    q = qd.cpu().numpy().astype(np.float64)
    e_rcp = float(np.max(np.abs(q * r.astype(np.float64) - 1.0)))
    print(f"ex2.approx max rel err {e_ex2:.3e} (bound {b_ex2:.3e}); rcp.approx {e_rcp:.3e} (bound {b_rcp:.3e})")
    assert e_ex2 < 0.5 * b_ex2
    assert e_rcp < 0.5 * b_rcp
    with pytest.raises(mgx.MgxError):
        mgx.mgx_eval_approx(ctx.ptr, 3, xd, yd)


def test_atan2_error_bound(ctx):
    """atan2f as the single-precision ray-set screen evaluates it stays within
    half the absolute bound its pixel certification takes, over random
    directions (all quadrants, up to 1e4 in ratio), the axes and the branch cut."""
    import torch

    import paper_2011_14998_gb300 as mgx

    rng = np.random.default_rng(4)
    n = 1 << 22
    ang = rng.uniform(-np.pi, np.pi, n)
    r = 10.0 ** rng.uniform(-3, 3, n)
    xs = (r * np.cos(ang)).astype(np.float32)
    ys = (r * np.sin(ang)).astype(np.float32)
    extra_x = np.array([1, -1, 0, 0, -1, -1, 1e-4, -1e-4, 3.0], np.float32)
    extra_y = np.array([0, 0, 1, -1, 1e-30, -1e-30, 1.0, 1.0, 1e-7], np.float32)
    xs, ys = np.concatenate([xs, extra_x]), np.concatenate([ys, extra_y])
    m = len(xs)
    xd = torch.from_numpy(np.concatenate([xs, ys])).cuda()
    yd = torch.empty(m, dtype=torch.float32, device="cuda")
    bound = mgx.mgx_eval_approx(ctx.ptr, 2, xd, yd)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.float64)
    ref = np.arctan2(ys.astype(np.float64), xs.astype(np.float64))
    err = np.abs(got - ref)
    err = np.minimum(err, 2 * np.pi - err)  # the branch cut: +pi and -pi are the same direction
    print(f"atan2f max abs err {err.max():.3e} (bound {bound:.3e})")
    assert err.max() < 0.5 * bound


def test_ex2_flushes_far_wings_to_zero(ctx):
    """2^x as the solve evaluates it is exactly +0 for every x <= -128 (a
    subnormal result, flushed): the single-precision solve skips the profile of
    samples whose every bin has a'^2 >= 128 and takes the continuum alone,
    which is then the same value bit for bit."""
    import torch

    import paper_2011_14998_gb300 as mgx

    x = np.concatenate([-np.linspace(128.0, 1000.0, 1 << 20), [-128.0, -np.inf, -3.0e38]]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, 1.0)
    mgx.mgx_eval_approx(ctx.ptr, 0, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.all(y == 0.0) and not np.any(np.signbit(y))


def test_eq2_near_ties_take_the_definitions_count(ctx, orc):
    """A dense two-point medium whose opacity puts Eq. 2's ratio within a few
    units of single-precision rounding of an integer on many bins: J of the
    single-precision form equals the oracle's to the FP32 tolerance (a
    sub-interval more or fewer would move it by far more), and some decisions
    were redone in double precision."""
    import paper_2011_14998_gb300 as mgx

    # three collinear points, origin in the middle, unit spacing; chi0 chosen so
    # that chi ds / dtau_max = 3 (1 + 2e-8) at line centre: between the float
    # neighbours of 3
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    off = np.array([0, 1, 3, 4])
    nbr = np.array([1, 0, 2, 1], np.int32)
    dtau_max = 0.5
    chi0 = 3.0 * dtau_max * (1.0 + 2e-8) - 1e-3
    m = dict(pos=pos, vel=np.zeros((3, 3)), nbr_off=off, nbr_idx=nbr, nu0=np.array([1e11]),
             chi0=np.full((3, 1), chi0), eta0=np.full((3, 1), 0.7), dvw=np.ones(3), chi_c=np.full(3, 1e-3),
             eta_c=np.full(3, 1e-3), n_freq=7, x_span=0.0, l_min=0, l_max=0)
    mid = ctx.load(m)
    rays = ctx.rays(mid)
    ctx.profile(True)
    u32 = ctx.solve_u(mid, 1, 2, precision=mgx.MGX_FP32, dtau_max=dtau_max)[0]
    prof = ctx.profile_read()
    ctx.profile(False)
    u64 = ctx.solve_u(mid, 1, 2, precision=mgx.MGX_FP64, dtau_max=dtau_max)[0]
    ctx.free(mid)
    uo = orc.OracleModel(m, rays=rays).solve_u(orc.params(dtau_max=dtau_max), [1])[0]
    assert j_rel_err(u64, uo)[0] < 1e-10
    assert j_rel_err(u32, uo)[0] < 1e-4
    assert prof["decisions_redone"] > 0


def test_fast_wind_far_wings_match_oracle(ctx, orc):
    """A wind three times faster (45 km/s) puts most traced points far in the
    wings of every bin, where the single-precision solve takes the continuum
    without the profile (velocity sampling off, so that the oracle stays
    quick): J of the FP32 form against the FP64 oracle (1e-4) on sampled
    origins and against the GPU FP64 form everywhere.  (Much faster winds
    leave the 1e-4 budget by the single-precision Doppler argument itself:
    at 300 km/s, |delta| / dv ~ 600 and its rounding alone moves J by 2e-4.)"""
    import synth

    import paper_2011_14998_gb300 as mgx

    m = synth.wind_model(1500, seed=61, n_freq=50, level=1, v_inf=45.0)
    mid = ctx.load(m)
    J32 = ctx.solve_J(mid, precision=mgx.MGX_FP32, dv_max=0.0)
    J32b = ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, dv_max=0.0)[0].cpu().numpy()
    J64 = ctx.solve_J(mid, precision=mgx.MGX_FP64, dv_max=0.0)
    rays = ctx.rays(mid)
    ctx.free(mid)
    origins = np.arange(0, 1500, 6)
    Jo = orc.OracleModel(m, rays=rays).solve_J(orc.params(dv_max=0.0), origins=origins)
    assert j_rel_err(J64[origins], Jo)[0] < 1e-10
    assert j_rel_err(J32[origins], Jo)[0] < 1e-4
    assert j_rel_err(J32, J64)[0] < 1e-4
    assert j_rel_err(J32b, J32)[0] < 1e-5
