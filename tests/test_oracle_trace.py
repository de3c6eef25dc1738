"""Pins of the oracle's tracer (Section 2.1, Fig. 2).

Exhaustive brute force on tiny meshes: every step of every traced half-ray is
re-derived from the neighbour list with NumPy, and the straight grid lines of a
Cartesian cube are checked against their exact projected distances.
"""
import numpy as np
import pytest


def _trace_brute(m, o, d):
    """Independent restatement of the next-point rule with NumPy."""
    pos, off, nbr = m["pos"], m["nbr_off"], m["nbr_idx"]
    c, zc, out = o, 0.0, []
    while True:
        nb = nbr[off[c]:off[c + 1]].astype(np.int64)
        delta = pos[nb] - pos[o]
        Z = (delta[:, 0] * d[0] + delta[:, 1] * d[1]) + delta[:, 2] * d[2]
        fwd = Z > zc
        if not fwd.any():
            return out
        e = delta - Z[:, None] * np.asarray(d)[None, :]
        q = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
        cand = np.where(fwd)[0]
        qmin = q[cand].min()
        best = int(nb[cand[q[cand] == qmin]].min())  # ties to the smaller index
        k = int(np.where(nb == best)[0][0])
        out.append((best, float(Z[k])))
        c, zc = best, float(Z[k])


def _check_mesh(orc, m, levels=(0, 1)):
    om = orc.OracleModel(m, l_min=0, l_max=0)
    n = len(m["pos"])
    edges = {(a, int(b)) for a in range(n) for b in m["nbr_idx"][m["nbr_off"][a]:m["nbr_off"][a + 1]]}
    for l in levels:
        dirs = orc.pix2vec(l, np.arange(orc.npix(l)))
        for o in range(n):
            for d in dirs:
                idx, Z = om.trace_half(o, d)
                ref = _trace_brute(m, o, d)
                assert [i for i, _ in ref] == list(idx)
                assert [z for _, z in ref] == list(Z)  # bit-exact
                assert np.all(np.diff(np.concatenate([[0.0], Z])) > 0)  # Z strictly increases
                prev = o
                for i in idx:  # every step follows an edge of the neighbour graph
                    assert (prev, int(i)) in edges
                    prev = int(i)


def test_trace_brute_grid3(orc):
    import synth

    m = synth.grid_model(3)
    _check_mesh(orc, m)


@pytest.mark.parametrize("n,seed", [(20, 1), (45, 2)])
def test_trace_brute_random(orc, n, seed):
    import synth

    m = synth.random_cloud(n, seed=seed)
    _check_mesh(orc, m)


def test_trace_straight_grid_lines(orc):
    import synth

    m = synth.grid_model(16)
    om = orc.OracleModel(m)
    d = orc.pix2vec(0, 4)
    assert list(d) == [1.0, 0.0, 0.0]  # base pixel 4 points exactly along +x
    x = np.arange(16) / 15.0
    for (j, k) in [(0, 0), (7, 3), (15, 15)]:
        o = (0 * 16 + j) * 16 + k
        idx, Z = om.trace_half(o, d)
        assert list(idx) == [(i * 16 + j) * 16 + k for i in range(1, 16)]
        assert np.array_equal(Z, x[1:] - x[0])
        # the opposite direction from the far face walks back
        o2 = (15 * 16 + j) * 16 + k
        idx2, Z2 = om.trace_half(o2, -d)
        assert list(idx2) == [(i * 16 + j) * 16 + k for i in range(14, -1, -1)]
        assert np.allclose(Z2, np.arange(1, 16) / 15.0, rtol=0, atol=1e-15)


def test_trace_boundary_point_has_empty_half(orc):
    import synth

    m = synth.grid_model(4)
    om = orc.OracleModel(m)
    d = orc.pix2vec(0, 4)
    o = (3 * 4 + 1) * 4 + 2  # on the x = 1 face
    idx, Z = om.trace_half(o, d)
    assert len(idx) == 0
