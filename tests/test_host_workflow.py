"""Host-side parts of the reduction workflow and of the experiments (Section
2.2.2, Section 3.2): re-meshing, barycentric mapping of J back to the full
mesh, the per-point error and its CDF, the feature standardisation, and the
dense-pair lookup of the adaptive-vs-dense comparison.  No GPU is used."""
import numpy as np
import pytest


def _csr_edges(off, nbr):
    return {(i, int(j)) for i in range(len(off) - 1) for j in nbr[off[i]:off[i + 1]]}


def test_delaunay_neighbours_of_a_tetrahedron_with_its_centre():
    # the four corners of a regular tetrahedron and its centre: the Delaunay
    # tetrahedralisation is the four tetrahedra around the centre, so every pair
    # of the five points is an edge (the complete graph)
    from paper_2011_14998_gb300.learned import delaunay_neighbours

    pos = np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [0.01, 0.02, 0.03]])
    off, nbr = delaunay_neighbours(pos)
    assert off[0] == 0 and off[-1] == 20
    assert _csr_edges(off, nbr) == {(i, j) for i in range(5) for j in range(5) if i != j}


def test_delaunay_neighbours_are_symmetric_sorted_and_cover_the_simplices():
    from scipy.spatial import Delaunay

    from paper_2011_14998_gb300.learned import delaunay_neighbours

    pos = np.random.default_rng(3).uniform(-1, 1, (300, 3))
    off, nbr = delaunay_neighbours(pos)
    edges = _csr_edges(off, nbr)
    assert all((j, i) in edges for i, j in edges)
    assert all(i != j for i, j in edges)
    for i in range(len(pos)):
        row = nbr[off[i]:off[i + 1]]
        assert np.all(np.diff(row) > 0)
    for s in Delaunay(pos).simplices:
        for a in range(4):
            for b in range(4):
                if a != b:
                    assert (int(s[a]), int(s[b])) in edges


def test_remesh_keeps_the_kept_points_fields():
    from paper_2011_14998_gb300.learned import remesh

    rng = np.random.default_rng(5)
    n = 200
    m = dict(name="cloud", pos=rng.uniform(-1, 1, (n, 3)), vel=rng.normal(size=(n, 3)), chi0=rng.uniform(1, 2, (n, 2)),
             eta0=rng.uniform(1, 2, (n, 2)), dvw=rng.uniform(0.5, 1, n), chi_c=rng.uniform(1, 2, n),
             eta_c=rng.uniform(1, 2, n), rho=rng.uniform(1, 2, n), T=rng.uniform(1, 2, n), n_freq=7)
    keep = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    r = remesh(m, keep)
    idx = np.flatnonzero(keep)
    for k in ("pos", "vel", "chi0", "eta0", "dvw", "chi_c", "eta_c", "rho", "T"):
        assert np.array_equal(r[k], m[k][idx])
    assert r["n_freq"] == 7
    assert len(r["nbr_off"]) == len(idx) + 1 and r["nbr_idx"].max() < len(idx)
    assert np.array_equal(r["sample"], np.arange(len(idx)))


def test_interpolate_is_exact_for_linear_fields_and_nearest_outside_the_hull():
    from paper_2011_14998_gb300.learned import interpolate

    rng = np.random.default_rng(7)
    src = rng.uniform(-1, 1, (400, 3))
    A = np.array([[1.0, -2.0], [0.5, 3.0], [-1.5, 0.25]])
    b = np.array([2.0, -1.0])
    values = src @ A + b
    inside = rng.uniform(-0.3, 0.3, (50, 3))  # well inside the hull of the cloud
    got = interpolate(src, values, inside)
    np.testing.assert_allclose(got, inside @ A + b, rtol=0, atol=1e-10)
    outside = np.array([[5.0, 0, 0], [0, -4.0, 0]])
    got = interpolate(src, values, outside)
    nn = [int(np.argmin(((src - p) ** 2).sum(1))) for p in outside]
    assert np.array_equal(got, values[nn])


def test_point_errors_average_over_the_bins_above_the_floor():
    from paper_2011_14998_gb300.learned import point_errors

    J = np.array([[1.0, 2.0, 1e-9], [4.0, 4.0, 4.0]])
    Ja = np.array([[1.1, 2.0, 5.0], [2.0, 4.0, 6.0]])
    # point 0: the third bin is below 1e-6 of the point's maximum and does not count
    np.testing.assert_allclose(point_errors(J, Ja), [0.05, 1.0 / 3.0], rtol=1e-14)
    assert point_errors(J, J).tolist() == [0.0, 0.0]


def test_error_cdf_steps_at_each_error():
    from paper_2011_14998_gb300.experiments import error_cdf

    err = np.array([0.0, 1e-9, 1e-3, 1e-3, 0.05, 30.0])
    edges, cdf = error_cdf(err, bins=900, lo=-8.0, hi=1.0)
    assert len(edges) == 900 and edges[-1] == pytest.approx(1.0)
    assert np.all(np.diff(cdf) >= 0) and cdf[-1] == pytest.approx(1.0)

    def at(x):  # fraction at or below the edge just above log10(x)
        return cdf[np.searchsorted(edges, np.log10(x) + 1e-9)]

    assert at(1e-8) == pytest.approx(2 / 6)  # zero and 1e-9 fall in the first bin
    assert at(1e-3) == pytest.approx(4 / 6)
    assert at(0.05) == pytest.approx(5 / 6)
    assert cdf[np.searchsorted(edges, np.log10(0.05)) - 2] == pytest.approx(4 / 6)


def test_standardizer():
    from paper_2011_14998_gb300.learned import Standardizer

    rng = np.random.default_rng(1)
    X = np.column_stack([rng.normal(3.0, 2.0, 500), np.full(500, 7.0)])
    Z = Standardizer(X)(X)
    assert Z.dtype == np.float32
    np.testing.assert_allclose(Z[:, 0].mean(), 0.0, atol=1e-6)
    np.testing.assert_allclose(Z[:, 0].std(), 1.0, rtol=1e-5)
    assert np.all(Z[:, 1] == 0.0)  # a constant feature stays finite (its spread is floored)


def test_dense_columns_cover_every_pixel_through_its_pair():
    import paper_2011_14998_gb300 as mgx
    from paper_2011_14998_gb300.experiments import _dense_columns

    mgx.build()
    lmax = 2
    npix = 12 * 4 ** lmax
    reps = [p for p in range(npix) if p < mgx.mgx_antipode(lmax, p)]  # one pixel per antipodal pair
    row = np.array([(lmax << 28) | p for p in reps], np.uint32)
    cols = _dense_columns(row, lmax)
    assert len(reps) == npix // 2
    for q in range(npix):
        rep = reps[cols[q]]
        assert q in (rep, mgx.mgx_antipode(lmax, rep))
