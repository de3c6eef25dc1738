"""Pins of the oracle's Hermitian (fourth-order) Feautrier solve (Section 2.1:
Auer 1976, third-order boundary conditions of Auer 1967).

* On a uniform grid the interior rows reduce to the textbook Numerov weights
  1/12, 10/12, 1/12: compared with a dense solve of that system written
  independently from the textbook form.
* A solution that is a symmetric quadratic in tau is reproduced exactly on
  random non-uniform grids (interior and boundary rows are exact for it).
* Against the closed form of a homogeneous slab the error falls by at least a
  factor 7 per halving of the increments: third order overall, the order of
  the boundary condition (the second-order scheme gives 4), on uniform and on
  randomly non-uniform grids, and is well below the second-order error.
* Deep inside an optically thick medium u = S; a one-point line gives I.
"""
import numpy as np
import pytest


def _numerov_uniform(M, h, S, I):
    """Textbook uniform-grid Numerov discretisation of u'' = u - S,
    (u_{i+1} - 2u_i + u_{i-1})/h^2 = (f_{i-1} + 10 f_i + f_{i+1})/12, f = u - S,
    closed by u' = u - I at both ends with u' = (u_1 - u_0)/h - h/2 f_0 - h/6 (f_1 - f_0)."""
    n = M + 1
    Amat = np.zeros((n, n))
    rhs = np.zeros(n)
    for i in range(1, M):
        Amat[i, i - 1] = 1 / h**2 - 1 / 12
        Amat[i, i] = -2 / h**2 - 10 / 12
        Amat[i, i + 1] = 1 / h**2 - 1 / 12
        rhs[i] = -(S[i - 1] + 10 * S[i] + S[i + 1]) / 12
    for e, nx in ((0, 1), (M, M - 1)):
        # (u_nx - u_e)/h - h/2 (u_e - S_e) - h/6 ((u_nx - S_nx) - (u_e - S_e)) - (u_e - I) = 0
        Amat[e, nx] = 1 / h - h / 6
        Amat[e, e] = -1 / h - h / 2 + h / 6 - 1
        rhs[e] = -h / 2 * S[e] + h / 6 * S[e] - h / 6 * S[nx] - I
    return np.linalg.solve(Amat, rhs)


@pytest.mark.parametrize("M,h", [(2, 0.3), (7, 0.1), (40, 0.05)])
def test_uniform_grid_is_numerov(orc, M, h):
    rng = np.random.default_rng(M)
    S = rng.uniform(0.2, 2.0, M + 1)
    I = 0.37
    u = orc.feautrier(np.full(M, h), S, 0, I_bdy=I, all_rows=True, order=4)
    ref = _numerov_uniform(M, h, S, I)
    assert np.allclose(u, ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_quadratic_solution_exact_on_nonuniform_grid(orc, seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(1, 30))
    dtau = rng.uniform(0.02, 0.5, M)
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    T = tau[-1]
    a, b = 1.3, 0.7
    x = tau - T / 2
    u_exact = a + b * x**2          # symmetric about the middle
    S = u_exact - 2 * b             # (1 - d2/dtau2) u = S
    I = u_exact[0] + b * T          # u - du/dtau at tau = 0 (and u + du/dtau at T)
    u = orc.feautrier(dtau, S, 0, I_bdy=I, all_rows=True, order=4)
    assert np.allclose(u, u_exact, rtol=0, atol=1e-11)


def _slab_error(orc, dtau, order):
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    T = tau[-1]
    io = len(dtau) // 2
    S = np.full(len(tau), 1.0)
    u = orc.feautrier(dtau, S, io, I_bdy=0.0, order=order)
    exact = 1.0 - 0.5 * (np.exp(-tau[io]) + np.exp(-(T - tau[io])))
    return abs(u - exact)


@pytest.mark.parametrize("jitter", [0.0, 0.4])
def test_fourth_order_convergence_on_homogeneous_slab(orc, jitter):
    rng = np.random.default_rng(3)
    base = 1.0 + jitter * rng.uniform(-1, 1, 8)  # shape of the grid, refined by halving
    errs4, errs2 = [], []
    for k in range(4):
        h = 0.4 / 2**k
        d = np.repeat(base, 2**k) * h
        errs4.append(_slab_error(orc, d, 4))
        errs2.append(_slab_error(orc, d, 2))
    ratios = [errs4[i] / errs4[i + 1] for i in range(3)]
    assert min(ratios) > 7.0, (errs4, ratios)
    assert max(errs2[i] / errs2[i + 1] for i in range(3)) < 4.1
    assert errs4[-1] < 0.2 * errs2[-1]


def test_thick_medium_and_single_point(orc):
    dtau = np.full(200, 0.4)
    S = np.full(201, 2.5)
    assert orc.feautrier(dtau, S, 100, I_bdy=0.0, order=4) == pytest.approx(2.5, abs=1e-12)
    assert orc.feautrier(np.zeros(0), np.array([3.0]), 0, I_bdy=0.8, order=4) == 0.8


def test_vanishing_increment_next_to_normal_ones(orc):
    # traced points can be 1e-17 apart in tau (grid lines along axis directions):
    # rows whose increments differ by more than a factor 64 take the second-order
    # weights, so the result stays finite and close to the slab solution, and it
    # is unchanged when S carries rounding-level noise (the compact weights would
    # amplify that noise by the increment ratio, 1e15 here)
    base = np.full(40, 0.05)
    d = np.concatenate([np.full(5, 2e-17), base])
    tau = np.concatenate([[0.0], np.cumsum(d)])
    S = np.ones(len(tau))
    io = 20
    exact = 1.0 - 0.5 * (np.exp(-tau[io]) + np.exp(-(tau[-1] - tau[io])))
    u = orc.feautrier(d, S, io, order=4)
    assert abs(u - exact) < 1e-4
    Sn = S * (1 + 1e-16 * np.random.default_rng(0).choice([-1.0, 1.0], len(S)))
    assert abs(orc.feautrier(d, Sn, io, order=4) - u) < 1e-12


def test_two_point_line_boundary_rows(orc):
    # M = 1: the two boundary rows alone; compare with their 2x2 dense solve
    h, S0, S1, I = 0.3, 1.2, 0.4, 0.1
    A = np.array([[2 / 3 + 2 / h + 2 / h**2, -(2 / h**2 - 1 / 3)],
                  [-(2 / h**2 - 1 / 3), 2 / 3 + 2 / h + 2 / h**2]])
    r = np.array([2 / 3 * S0 + 1 / 3 * S1 + 2 * I / h, 2 / 3 * S1 + 1 / 3 * S0 + 2 * I / h])
    u = orc.feautrier([h], [S0, S1], 0, I_bdy=I, all_rows=True, order=4)
    assert np.allclose(u, np.linalg.solve(A, r), rtol=1e-13)


def test_solve_J_order_parameter(orc):
    import synth

    m = synth.grid_model(6, n_freq=5)
    om = orc.OracleModel(m)
    J2 = om.solve_J(orc.params(order=2))
    J4 = om.solve_J(orc.params(order=4))
    assert J2.shape == J4.shape
    assert not np.array_equal(J2, J4)
    assert np.allclose(J2, J4, rtol=2e-2)  # both discretise the same problem
    with pytest.raises(ValueError):
        orc.params(order=3)


def test_grid_J_closed_form_hermitian(orc):
    # the 16^3 homogeneous cube: the axis rays carry points 1e-17 apart (libm's
    # cos(pi/2) is not 0), whose rows take the second-order weights, so J
    # converges at second order here, below the second-order scheme's error
    import synth

    from test_oracle_solver import _grid_closed_form

    m = synth.grid_model(16)
    om = orc.OracleModel(m)
    origins = np.arange(0, 4096, 37)
    ref = _grid_closed_form(orc, m, om, None, origins)
    for dtm in (0.2, 0.1, 0.05):
        e4 = np.abs(om.solve_J(orc.params(dtau_max=dtm, order=4), origins=origins) - ref).max()
        e2 = np.abs(om.solve_J(orc.params(dtau_max=dtm), origins=origins) - ref).max()
        assert e4 < 0.6 * e2, (dtm, e4, e2)
    assert e4 <= 2e-5
