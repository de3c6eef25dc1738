"""Input generators: the octree leaves tile the box, the leaf adjacency equals a
brute-force closed-cube intersection test, and the batch generator draws the
stated sizes, generators and line layout."""
import numpy as np

import synth


def _cubes(m, box):
    h = box / 2.0 ** m["level"]
    return m["pos"] - h[:, None] / 2, m["pos"] + h[:, None] / 2


def test_octree_leaves_tile_the_box():
    m = synth.octree_model(3000, seed=7, hi_level=6)
    box = 1000.0
    h = box / 2.0 ** m["level"]
    assert np.isclose((h ** 3).sum(), box ** 3, rtol=1e-12)
    assert m["level"].min() >= 3 and m["level"].max() <= 6
    assert abs(len(m["pos"]) - 3000) <= 0.05 * 3000
    lo, hi = _cubes(m, box)
    assert (lo >= -box / 2 - 1e-9).all() and (hi <= box / 2 + 1e-9).all()


def test_octree_adjacency_is_closed_cube_contact():
    m = synth.octree_model(400, seed=8, hi_level=5)
    lo, hi = _cubes(m, 1000.0)
    n = len(lo)
    touch = np.all((lo[:, None, :] <= hi[None, :, :] + 1e-9) & (lo[None, :, :] <= hi[:, None, :] + 1e-9), axis=2)
    overlap = np.all((lo[:, None, :] < hi[None, :, :] - 1e-9) & (lo[None, :, :] < hi[:, None, :] - 1e-9), axis=2)
    np.fill_diagonal(touch, False)
    np.fill_diagonal(overlap, False)
    assert not overlap.any()  # leaves never overlap
    A = np.zeros((n, n), bool)
    for i in range(n):
        A[i, m["nbr_idx"][m["nbr_off"][i]:m["nbr_off"][i + 1]]] = True
    assert np.array_equal(A, touch)
    for i in range(n):  # rows sorted ascending, no duplicates
        row = m["nbr_idx"][m["nbr_off"][i]:m["nbr_off"][i + 1]]
        assert np.all(np.diff(row) > 0)


def test_octree_velocity_field_rms():
    m = synth.octree_model(2000, seed=9, hi_level=5)
    assert np.allclose(m["vel"].std(0), 2.0, rtol=1e-12)
    m2 = synth.octree_model(2000, seed=9, hi_level=5, velocity="iid")
    assert abs(m2["vel"].std() - 2.0) < 0.1


def test_batch_generator_layout():
    ms = synth.batch_models(n_models=6, seed=11, n_min=300, n_max=1500, n_lines=4, n_freq=20)
    assert len(ms) == 6
    names = [m["name"] for m in ms]
    assert names[0].startswith("grid") and names[1].startswith("wind") and names[2].startswith("octree")
    for m in ms:
        n = len(m["pos"])
        assert m["chi0"].shape == (n, 4) and m["eta0"].shape == (n, 4) and len(m["nu0"]) == 4
        assert (m["l_min"], m["l_max"], m["n_freq"]) == (0, 3, 20)
        # line centres several hundred widths apart (1e-3 relative = 300 km/s)
        assert np.diff(m["nu0"]).min() / m["nu0"][0] * 299792.458 > 200 * m["dvw"].max()
        assert 200 <= n <= 2000
