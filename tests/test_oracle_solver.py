"""Pins of the oracle's line mapping and Feautrier solver (Sections 2.1.1-2.1.3, Eqs. 1-3).

The discretised system is assembled here from the equations and solved with a
dense LU; the homogeneous slab is compared with its closed form and its
second-order convergence; optically thick media must give J = S; the profile
argument is checked in 50-digit arithmetic against the frequency-space
definition; the sub-division against Eq. 2's guarantee and the trapezoid sums.
"""
import math

import numpy as np
import pytest

from helpers import line_model


def _dense_system(dtau, S, I):
    M = len(dtau)
    A = np.zeros((M + 1, M + 1))
    b = np.array(S, dtype=np.float64).copy()
    t0 = dtau[0]
    A[0, 0] = 1 + 2 / t0 + 2 / t0 ** 2
    A[0, 1] = -2 / t0 ** 2
    b[0] += 2 * I / t0
    for i in range(1, M):
        tm, tp = dtau[i - 1], dtau[i]
        a = 2 / (tm * (tm + tp))
        c = 2 / (tp * (tm + tp))
        A[i, i - 1], A[i, i], A[i, i + 1] = -a, 1 + a + c, -c
    tl = dtau[-1]
    A[M, M] = 1 + 2 / tl + 2 / tl ** 2
    A[M, M - 1] = -2 / tl ** 2
    b[M] += 2 * I / tl
    return A, b


@pytest.mark.parametrize("M", [1, 2, 3, 7, 20, 50])
def test_feautrier_equals_dense_solve(orc, M):
    rng = np.random.default_rng(M)
    for _ in range(5):
        dtau = np.exp(rng.uniform(np.log(0.01), np.log(5.0), M))
        S = rng.uniform(0.0, 2.0, M + 1)
        I = rng.uniform(0.0, 1.0)
        A, b = _dense_system(dtau, S, I)
        ref = np.linalg.solve(A, b)
        u = orc.feautrier(dtau, S, 0, I, all_rows=True)
        assert np.allclose(u, ref, rtol=1e-11, atol=0)
        for io in range(M + 1):
            assert orc.feautrier(dtau, S, io, I) == pytest.approx(ref[io], rel=1e-11)


def test_feautrier_single_point_is_boundary_intensity(orc):
    assert orc.feautrier(np.zeros(0), np.array([3.0]), 0, 0.25) == 0.25


def _slab_error(orc, T, n, S=1.0):
    dtau = np.full(n, T / n)
    u = orc.feautrier(dtau, np.full(n + 1, S), 0, 0.0, all_rows=True)
    tau = np.linspace(0, T, n + 1)
    exact = S * (1 - 0.5 * (np.exp(-tau) + np.exp(-(T - tau))))
    return np.abs(u - exact).max()


def test_homogeneous_slab_second_order(orc):
    # (1 - d2/dtau2) u = S on [0, T], no incoming light: u = S (1 - (e^-tau + e^-(T-tau))/2)
    errs = [_slab_error(orc, 3.0, n) for n in (15, 30, 60, 120)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios
    assert errs[-1] < 2e-4


def test_boundary_light_propagates(orc):
    T, n, I = 2.0, 400, 0.7
    dtau = np.full(n, T / n)
    u = orc.feautrier(dtau, np.zeros(n + 1), 0, I, all_rows=True)
    tau = np.linspace(0, T, n + 1)
    assert np.allclose(u, I * 0.5 * (np.exp(-tau) + np.exp(-(T - tau))), atol=5e-6)


def test_optically_thick_gives_source(orc):
    T, n, S = 60.0, 600, 0.37
    u = orc.feautrier(np.full(n, T / n), np.full(n + 1, S), n // 2, 0.0)
    assert abs(u - S) < 1e-6


def test_bin_grid(orc):
    xs = [orc.bin_x(31, 4.0, k) for k in range(31)]
    assert xs[0] == -4.0 and xs[-1] == 4.0 and xs[15] == 0.0
    assert np.allclose(np.diff(xs), 8.0 / 30, rtol=1e-14)
    assert orc.bin_x(1, 4.0, 0) == 0.0


def test_profile_argument_50_digits(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    c = mp.mpf("299792.458")
    rng = np.random.default_rng(7)
    for _ in range(300):
        nu_l = 115.2712018e9 * (1 + rng.uniform(-1e-3, 1e-3))
        nu_lp = 115.2712018e9 * (1 + rng.uniform(-1e-3, 1e-3)) if rng.uniform() < 0.5 else nu_l
        x, dvo, delta, dv = rng.uniform(-4, 4), rng.uniform(0.2, 2), rng.uniform(-30, 30), rng.uniform(0.2, 2)
        nu = mp.mpf(nu_l) * (1 + mp.mpf(x) * mp.mpf(dvo) / c)  # bin frequency, origin frame
        nup = nu * (1 + mp.mpf(delta) / c)  # as seen by the moving point
        ref = (nup - mp.mpf(nu_lp)) / (mp.mpf(nu_lp) * mp.mpf(dv) / c)
        got = orc.profile_arg(nu_l, nu_lp, x, dvo, delta, dv)
        assert abs(got - float(ref)) <= 1e-9 * max(1.0, abs(float(ref))), (got, float(ref))


def test_subdivision_eq2(orc):
    rng = np.random.default_rng(3)
    for _ in range(50):
        m = rng.integers(2, 12)
        s = np.cumsum(rng.uniform(0.01, 1.0, m))
        chi = np.exp(rng.uniform(-3, 3, m))
        eta = chi * rng.uniform(0.1, 2, m)
        io = int(rng.integers(0, m))
        dtm = rng.uniform(0.05, 1.0)
        dtau, S, io2 = orc.subdivide(s, chi, eta, io, dtm)
        assert np.all(dtau <= dtm * (1 + 1e-12))  # Eq. 2 guarantees dtau <= dtau_max
        # per original interval: the count is Eq. 2's n_inter, the sum is the trapezoid
        k = 0
        for i in range(m - 1):
            ni = max(1, math.ceil(max(chi[i], chi[i + 1]) * (s[i + 1] - s[i]) / dtm))
            tot = dtau[k:k + ni].sum()
            assert tot == pytest.approx((s[i + 1] - s[i]) * (chi[i] + chi[i + 1]) / 2, rel=1e-12)
            if i + 1 == io:
                assert io2 == k + ni
            k += ni
            assert S[k] == pytest.approx(eta[i + 1] / chi[i + 1], rel=1e-15)
        assert k == len(dtau)
        if io == 0:
            assert io2 == 0


def test_velocity_sampling_counts(orc):
    # pair of base pixel 4 (+x) at the middle point: backward point 0 (direction -x),
    # forward point 2 (+x).  delta_0 = (v_0 - v_1).(-x), delta_2 = (v_2 - v_1).(+x)
    m = line_model(vel_a=-2.0, vel_b=0.9)
    om = orc.OracleModel(m, rays=np.zeros((3, 6), np.uint32))
    ray = np.uint32(4)
    assert orc.antipode(0, 4) == 6
    # dv_max = 1/3 of the width 1 km/s: |2 - 0| -> ceil(6) = 6 parts, |0.9 - 0| -> 3 parts
    mv, io = om.vline_size(1, ray, orc.params(dv_max=1 / 3))
    assert (mv, io) == (1 + 6 + 3, 6)
    mv, io = om.vline_size(1, ray, orc.params(dv_max=0.0))  # sampling off
    assert (mv, io) == (3, 1)
    # the samples are equally spaced in s: with the line switched off the optical
    # depth of every sub-interval is the continuum opacity times its length
    m["chi0"] = np.zeros((3, 1))
    m["eta0"] = np.zeros((3, 1))
    om = orc.OracleModel(m, rays=np.zeros((3, 6), np.uint32))
    dtau, S, io = om.pair_line(1, ray, 0, 1, orc.params(dv_max=1 / 3, dtau_max=100.0))
    assert len(dtau) == 9 and io == 6
    assert np.allclose(dtau[:6], 1e-3 / 6, rtol=1e-13) and np.allclose(dtau[6:], 1e-3 / 3, rtol=1e-13)


def test_static_medium_line_mapping(orc):
    # No motion: the Doppler factor is exactly one, so the profile argument of a
    # line at its own bins is the rounded x dv_o / dv, and velocity sampling
    # inserts nothing (a pair line is the traced points plus the origin).
    rng = np.random.default_rng(11)
    for _ in range(200):
        nu, x, dvo, dv = 115.2712018e9 * rng.uniform(0.5, 2), rng.uniform(-5, 5), rng.uniform(0.1, 3), rng.uniform(0.1, 3)
        assert orc.profile_arg(nu, nu, x, dvo, 0.0, dv) == (x * dvo) / dv
    import synth

    m = synth.grid_model(6, level=1)
    om = orc.OracleModel(m)
    for o in (0, 43, 100, 215):
        for ray in om.rays[o]:
            d = orc.pix2vec(int(ray >> 28), int(ray & 0x0FFFFFFF))
            nb, nf = len(om.trace_half(o, -d)[0]), len(om.trace_half(o, d)[0])
            assert om.vline_size(o, ray, orc.params(dv_max=1 / 3)) == (nb + nf + 1, nb)


def test_velocity_count_at_a_near_tie(orc):
    # Section 2.1.1: an interval is split into ceil(|jump| / limit) parts.  Origin
    # v = 0.7, forward neighbour v = 2.7000001586834803 (direction +x), limit
    # 1/3 of the unit Doppler width: the jump is 2.00000015868... = 6.0000005
    # limits, so 7 parts (6 interpolated samples), although the jump of the
    # velocities rounded to single precision is exactly 6 limits.
    m = line_model(vel_a=0.7, vel_b=2.7000001586834803)
    m["vel"][1, 0] = 0.7
    om = orc.OracleModel(m, rays=np.zeros((3, 6), np.uint32))
    ray = np.uint32(4)
    assert om.vline_size(1, ray, orc.params(dv_max=1 / 3)) == (2 + 7, 1)
    # an exact multiple of the limit is not split further: jump 2.0 = 6 limits of 1/3
    m2 = line_model(vel_a=0.7, vel_b=2.0 + 0.5)
    m2["vel"][1, 0] = 0.5
    om2 = orc.OracleModel(m2, rays=np.zeros((3, 6), np.uint32))
    assert om2.vline_size(1, ray, orc.params(dv_max=0.25)) == (2 + 8, 1)


def _grid_closed_form(orc, m, om, params, origins):
    """J of the homogeneous S = 1 cube: sum over pairs 2 w (1 - (e^-tau+ + e^-tau-)/2),
    tau = chi(x) times the traced extent of each half-ray."""
    x = np.array([orc.bin_x(m["n_freq"], m["x_span"], k) for k in range(m["n_freq"])])
    chi = m["chi0"][0, 0] * np.exp(-x * x) + m["chi_c"][0]
    J = np.zeros((len(origins), len(x)))
    for qi, o in enumerate(origins):
        for ray in om.rays[o]:
            l, p = int(ray >> 28), int(ray & 0x0FFFFFFF)
            d = orc.pix2vec(l, p)
            _, Zf = om.trace_half(o, d)
            _, Zb = om.trace_half(o, -d)
            zf = Zf[-1] if len(Zf) else 0.0
            zb = Zb[-1] if len(Zb) else 0.0
            J[qi] += 2 / (12 * 4 ** l) * (1 - 0.5 * (np.exp(-chi * zf) + np.exp(-chi * zb)))
    return J


def test_grid_J_closed_form_and_convergence(orc):
    import synth

    m = synth.grid_model(16)
    om = orc.OracleModel(m)
    origins = np.arange(0, 4096, 37)
    ref = _grid_closed_form(orc, m, om, None, origins)
    errs = []
    for dtm in (0.2, 0.1, 0.05):
        J = om.solve_J(orc.params(dtau_max=dtm), origins=origins)
        errs.append(np.abs(J - ref).max())
    assert errs[-1] <= 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_thick_medium_J_equals_S(orc):
    import synth

    m = synth.grid_model(6, chi_line=3000.0, n_freq=3, x_span=0.5)
    m["eta0"] = 0.7 * m["chi0"]
    m["eta_c"] = 0.7 * m["chi_c"]
    om = orc.OracleModel(m)
    inner = [((i * 6 + j) * 6 + k) for i in range(1, 5) for j in range(1, 5) for k in range(1, 5)]
    J = om.solve_J(orc.params(dtau_max=1.0), origins=inner)
    assert np.abs(J - 0.7).max() < 1e-6


def test_J_weights_sum_to_one(orc):
    # constant S, I = S everywhere, any opacity: u = S on every ray, J = S (Eq. 3, 4)
    import synth

    m = synth.random_cloud(30, seed=4, l_min=0, l_max=2)
    m["eta0"] = 0.5 * m["chi0"]
    m["eta_c"] = 0.5 * m["chi_c"]
    om = orc.OracleModel(m)
    J = om.solve_J(orc.params(I_bdy=0.5))
    assert np.allclose(J, 0.5, rtol=1e-12)


def test_subdivision_count_at_the_ceiling(orc):
    # Eq. 2: n_inter = ceil(chi_max ds / dtau_max).  chi (5 + 5e-10) ds 0.2 /
    # dtau_max 0.5 is just above 2 in double precision -> 3 sub-intervals;
    # chi = 5 gives exactly 2 -> 2 sub-intervals; the sub-interval optical
    # depths sum to the trapezoid of the interval either way.
    s = np.array([0.0, 0.2])
    chi_a = np.array([5.0 + 5e-10, 5.0 + 5e-10])
    chi_b = np.array([5.0, 5.0])
    da, _, _ = orc.subdivide(s, chi_a, chi_a, 0, 0.5)
    db, _, _ = orc.subdivide(s, chi_b, chi_b, 0, 0.5)
    assert len(da) == 3 and len(db) == 2
    assert da.sum() == pytest.approx(0.2 * chi_a[0], rel=1e-15)
    assert db.sum() == pytest.approx(0.2 * chi_b[0], rel=1e-15)
