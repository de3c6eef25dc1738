"""Property tests of the oracle on random small inputs (hypothesis): the HEALPix
nested hierarchy and round trip, the tracer's defining rule checked by an
exhaustive scan, the Feautrier elimination against a dense solve of the same
system, Eq. 2's guarantee that no sub-interval exceeds dtau_max, and the
reduction criterion's ranges (Eqs. 6-8).  CPU only."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import HealthCheck, given, settings  # noqa: E402

from helpers import oracle_model_of  # noqa: E402

SETTINGS = dict(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])

unit = st.tuples(*[st.floats(-1.0, 1.0, allow_nan=False)] * 3).filter(lambda v: 0.1 < np.linalg.norm(v))


@settings(**SETTINGS)
@given(v=unit, l=st.integers(1, 8))
def test_healpix_nested_parent_and_round_trip(orc, v, l):
    d = np.asarray(v) / np.linalg.norm(v)
    p = int(orc.vec2pix(l, d)[0])
    assert 0 <= p < 12 * 4 ** l
    assert int(orc.vec2pix(l - 1, d)[0]) == p >> 2  # the parent pixel contains the direction too
    assert int(orc.vec2pix(l, orc.pix2vec(l, p))[0]) == p
    q = orc.antipode(l, p)
    assert int(orc.vec2pix(l, -orc.pix2vec(l, p))[0]) == q


def _tracer_case(seed, n):
    from paper_2011_14998_gb300.learned import delaunay_neighbours

    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1, 1, (n, 3))
    off, nbr = delaunay_neighbours(pos)
    return pos, off, nbr


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31), n=st.integers(12, 60), v=unit, o=st.integers(0, 10 ** 6))
def test_tracer_rule_by_exhaustive_scan(orc, seed, n, v, o):
    pos, off, nbr = _tracer_case(seed, n)
    o %= n
    d = np.asarray(v) / np.linalg.norm(v)
    idx, Z = oracle_model_of(orc, pos, off, nbr).trace_half(o, d)
    xo = pos[o]
    c, zc = o, 0.0
    for k in range(len(idx) + 1):
        best, qbest, zbest = -1, 0.0, 0.0
        for nb in nbr[off[c]:off[c + 1]]:
            dx, dy, dz = pos[nb] - xo
            zn = (dx * d[0] + dy * d[1]) + dz * d[2]
            if not zn > zc:
                continue
            ex, ey, ez = dx - zn * d[0], dy - zn * d[1], dz - zn * d[2]
            q = (ex * ex + ey * ey) + ez * ez
            if best < 0 or q < qbest or (q == qbest and nb < best):
                best, qbest, zbest = int(nb), q, zn
        if k == len(idx):
            assert best == -1  # the half-ray ends where no neighbour lies further along
            break
        assert best == idx[k] and zbest == Z[k] and Z[k] > zc
        c, zc = best, zbest


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31), M=st.integers(1, 30), I_bdy=st.floats(0.0, 2.0))
def test_feautrier_equals_dense_solve(orc, seed, M, I_bdy):
    rng = np.random.default_rng(seed)
    dtau = 10.0 ** rng.uniform(-3, 1, M)
    S = rng.uniform(0.1, 2.0, M + 1)
    io = int(rng.integers(0, M + 1))
    # the second-order system u'' = u - S with boundary rows u' = +-(u - I)
    A = np.zeros((M + 1, M + 1))
    b = S.copy()
    for i in range(1, M):
        hm, hp = dtau[i - 1], dtau[i]
        hb = 0.5 * (hm + hp)
        A[i, i - 1] = -1.0 / (hm * hb)
        A[i, i + 1] = -1.0 / (hp * hb)
        A[i, i] = 1.0 + 1.0 / (hm * hb) + 1.0 / (hp * hb)
    for i, h, j in ((0, dtau[0], 1), (M, dtau[-1], M - 1)):
        A[i, i] = 1.0 + 2.0 / h + 2.0 / (h * h)
        A[i, j] = -2.0 / (h * h)
        b[i] = S[i] + 2.0 * I_bdy / h
    u = np.linalg.solve(A, b)
    got = orc.feautrier(dtau, S, io, I_bdy=I_bdy)
    assert got == pytest.approx(u[io], rel=1e-9, abs=1e-12)


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31), m=st.integers(2, 20), dtau_max=st.floats(0.05, 3.0))
def test_eq2_sub_intervals_respect_dtau_max(orc, seed, m, dtau_max):
    rng = np.random.default_rng(seed)
    s = np.cumsum(rng.uniform(0.01, 2.0, m))
    chi = 10.0 ** rng.uniform(-2, 1.5, m)
    eta = chi * rng.uniform(0.5, 2.0, m)
    dtau, S, io = orc.subdivide(s, chi, eta, m // 2, dtau_max)
    # every trapezoid increment stays within dtau_max (Eq. 2's guarantee; chi is
    # linear on each sub-interval, so its largest value bounds the mean)
    assert np.all(dtau <= dtau_max * (1 + 1e-12))
    assert dtau.sum() == pytest.approx(np.sum(0.5 * (chi[1:] + chi[:-1]) * np.diff(s)), rel=1e-12)
    assert np.all(np.isfinite(S)) and len(S) == len(dtau) + 1


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31), n=st.integers(5, 80), f_small=st.floats(0.1, 1.0),
       f_large=st.floats(1.0, 4.0), G=st.floats(0.0, 1.0))
def test_reduction_ranges(orc, seed, n, f_small, f_large, G):
    pos, off, nbr = _tracer_case(seed, n)
    rng = np.random.default_rng(seed + 1)
    f = 10.0 ** rng.uniform(-3, 3, n)
    Gf, L, ell, keep = orc.reduce(pos, off, nbr, f, f_small, f_large, G, seed)
    assert np.all((Gf >= 0) & (Gf <= 1))  # Eq. 6
    for i in range(n):
        nb = nbr[off[i]:off[i + 1]]
        assert L[i] == pytest.approx(np.mean(np.linalg.norm(pos[nb] - pos[i], axis=1)), rel=1e-12)  # Eq. 8
        assert ell[i] == pytest.approx(L[i] * (f_small if Gf[i] >= G else f_large), rel=1e-12)  # Eq. 7
    assert set(np.unique(keep)) <= {0, 1}
