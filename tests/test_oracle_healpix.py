"""Pins of the oracle's HEALPix and adaptive ray set (Section 2.1.3, Eq. 4, Fig. 1).

Everything here is checked against facts that the paper or Gorski et al. (2005)
fix, not against the oracle itself: pixel counts, the geometry of the 12 base
pixels, the ring closed forms, nested parenthood, equal areas, the paper's ray
counts (552 adaptive, 3072 dense) and weights that sum to one.
"""
import math

import numpy as np
import pytest


def test_pixel_counts(orc):
    for l in range(9):
        assert orc.npix(l) == 12 * 4 ** l


def test_base_pixel_geometry(orc):
    # Gorski et al. (2005) Fig. 3: faces 0-3 north (z = 2/3), 4-7 equator, 8-11 south
    for f in range(12):
        v = orc.pix2vec(0, f)
        z = v[2]
        phi = math.atan2(v[1], v[0]) % (2 * math.pi)
        if f < 4:
            assert z == pytest.approx(2 / 3, abs=1e-15)
            assert phi == pytest.approx(math.pi / 4 + f * math.pi / 2, abs=1e-14)
        elif f < 8:
            assert z == pytest.approx(0.0, abs=1e-15)
            assert phi == pytest.approx(((f - 4) * math.pi / 2) % (2 * math.pi), abs=1e-14)
        else:
            assert z == pytest.approx(-2 / 3, abs=1e-15)
            assert phi == pytest.approx(math.pi / 4 + (f - 8) * math.pi / 2, abs=1e-14)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_ring_closed_forms(orc, l):
    ns = 2 ** l
    v = orc.pix2vec(l, np.arange(orc.npix(l)))
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    z = v[:, 2]
    phi = np.arctan2(v[:, 1], v[:, 0]) % (2 * np.pi)
    for i in range(1, 4 * ns):
        if i < ns:
            zi, nring, dphi, off = 1 - i * i / (3 * ns * ns), 4 * i, np.pi / (2 * i), 0.5
        elif i <= 3 * ns:
            s = 1 if (i - ns) % 2 == 0 else 0
            zi, nring, dphi, off = 4 / 3 - 2 * i / (3 * ns), 4 * ns, np.pi / (2 * ns), s / 2
        else:
            k = 4 * ns - i
            zi, nring, dphi, off = -(1 - k * k / (3 * ns * ns)), 4 * k, np.pi / (2 * k), 0.5
        sel = np.abs(z - zi) < 1e-12
        assert sel.sum() == nring, (i, sel.sum(), nring)
        # phi = dphi (j - off), j = 1..nring
        j = phi[sel] / dphi + off
        assert np.allclose(j, np.round(j), atol=1e-9)
        jj = np.sort((np.round(j).astype(np.int64) - 1) % nring)  # phi is periodic
        assert np.array_equal(jj, np.arange(nring))


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 5])
def test_round_trip(orc, l):
    p = np.arange(orc.npix(l))
    assert np.array_equal(orc.vec2pix(l, orc.pix2vec(l, p)), p)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_nested_parenthood(orc, l):
    p = np.arange(orc.npix(l))
    assert np.array_equal(orc.vec2pix(l - 1, orc.pix2vec(l, p)), p >> 2)


def test_equal_area(orc):
    # isotropic directions fall uniformly into the 192 pixels of level 2
    rng = np.random.default_rng(11)
    d = rng.normal(size=(200000, 3))
    cnt = np.bincount(orc.vec2pix(2, d), minlength=192)
    exp = len(d) / 192
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    # chi-square with 191 dof: mean 191, sd ~ 19.5; 191 + 6 sd
    assert chi2 < 310, chi2


def test_vec2pix_contains_direction(orc):
    # a direction lies closer to its own pixel centre than the pixel's diameter
    rng = np.random.default_rng(3)
    d = rng.normal(size=(5000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for l in (1, 3):
        c = orc.pix2vec(l, orc.vec2pix(l, d))
        ang = np.arccos(np.clip((c * d).sum(1), -1, 1))
        assert ang.max() < 2.5 * math.sqrt(4 * math.pi / orc.npix(l))


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_antipodes(orc, l):
    for p in range(orc.npix(l)):
        a = orc.antipode(l, p)
        assert a != p
        assert orc.antipode(l, a) == p
        assert np.allclose(orc.pix2vec(l, a), -orc.pix2vec(l, p), atol=1e-14)


def _desc(l, p, lmax):
    sh = 2 * (lmax - l)
    return set(range(p << sh, (p + 1) << sh))


@pytest.mark.parametrize("lmin,lmax,nrays", [(1, 4, 552), (4, 4, 3072), (0, 3, 138), (0, 0, 12),
                                             (2, 2, 192)])
def test_rayset_counts_and_weights(orc, lmin, lmax, nrays):
    import synth

    assert 2 * orc.rayset_npairs(lmin, lmax) == nrays
    m = synth.random_cloud(60, seed=5)
    rays = orc.rayset(m["pos"], lmin, lmax, m["sample"])
    assert rays.shape == (60, nrays // 2)  # the same number of rays at every point
    lev = (rays >> 28).astype(np.int64)
    w = 1.0 / (12.0 * 4.0 ** lev)
    assert np.allclose(2 * w.sum(1), 1.0, atol=1e-14)  # Eq. 4, sum over rays = 1
    # each ray set partitions the sphere: the finest-level descendants of all rays
    # and of their antipodes cover every finest pixel exactly once
    for o in range(0, 60, 13):
        cover = []
        for r in rays[o]:
            l, p = int(r >> 28), int(r & 0x0FFFFFFF)
            assert p < orc.antipode(l, p)
            cover += list(_desc(l, p, lmax)) + list(_desc(l, orc.antipode(l, p), lmax))
        assert sorted(cover) == list(range(orc.npix(lmax)))


def _rayset_brute(orc, pos, o, sample, lmin, lmax):
    """Independent restatement: counts taken at every level directly (no downgrade)."""
    d = pos[[j for j in sample if j != o]] - pos[o]
    d = d[np.any(d != 0, axis=1)]
    cand = sorted({min(p, orc.antipode(lmin, p)) for p in range(orc.npix(lmin))})
    rays = []
    for l in range(lmin, lmax):
        cnt = np.bincount(orc.vec2pix(l, d), minlength=orc.npix(l))
        score = {p: int(cnt[p] + cnt[orc.antipode(l, p)]) for p in cand}
        order = sorted(cand, key=lambda p: (-score[p], p))
        half = len(order) // 2
        rays += [(l, p) for p in order[half:]]
        cand = sorted({min(c, orc.antipode(l + 1, c)) for p in order[:half]
                       for c in range(4 * p, 4 * p + 4)})
    rays += [(lmax, p) for p in cand]
    return sorted((l << 28) | p for l, p in rays)


def test_rayset_against_brute_force(orc):
    import synth

    m = synth.random_cloud(50, seed=9)
    for lmin, lmax in [(0, 2), (1, 3)]:
        rays = orc.rayset(m["pos"], lmin, lmax, m["sample"])
        for o in range(0, 50, 7):
            assert list(rays[o]) == _rayset_brute(orc, m["pos"], o, m["sample"], lmin, lmax)


def test_rayset_follows_point_density(orc):
    # points concentrated in +z: the refined (finer) rays of the origin point there
    rng = np.random.default_rng(1)
    pos = np.vstack([[0.0, 0.0, 0.0], rng.normal([0, 0, 5], 0.5, (400, 3)),
                     rng.normal(0, 5, (40, 3))])
    rays = orc.rayset(pos, 0, 2, np.arange(len(pos), dtype=np.int32))[0]
    fine = [r for r in rays if (r >> 28) == 2]
    dirs = orc.pix2vec(2, np.array([r & 0x0FFFFFFF for r in fine]))
    assert np.abs(dirs[:, 2]).mean() > 0.5  # fine pairs are along the z axis
