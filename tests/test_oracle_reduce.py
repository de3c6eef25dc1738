"""Pins of the oracle's mesh-reduction criterion (Section 2.2.2, Eqs. 6-8, Table 1).

Hand-computed values on a 4-point graph, the range Gf in [0, 1] that Eq. 6
guarantees, published SplitMix64 outputs (Steele, Lea & Flood 2014) for the
thinning coin, and the thinning rate (L/ell)^3 in distribution.
"""
import math

import numpy as np
import pytest


def test_splitmix64_published_outputs(orc):
    # SplitMix64 started from state 0 gives 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    # 0x06C45D188009454F; the uniform is the top 53 bits
    for i, z in enumerate([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]):
        assert orc.uniform01(0, i) == (z >> 11) / 2.0 ** 53


def test_four_point_graph(orc):
    # square of side 1 and 2 in the plane, a path graph 0-1-2-3
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.0, 2.0, 0], [0.0, 2.0, 0]])
    off = np.array([0, 1, 3, 5, 6])
    nbr = np.array([1, 0, 2, 1, 3, 2], np.int32)
    f = np.array([1.0, 3.0, 3.0, 0.0])
    Gf, L, ell, keep = orc.reduce(pos, off, nbr, f, 0.9, 2.1, 0.1, seed=1)
    assert Gf == pytest.approx([0.5, 0.5, 1.0, 1.0])  # |1-3|/4, max(2/4, 0), |3-0|/3, 3/3
    assert L == pytest.approx([1.0, 1.5, 1.5, 1.0])
    assert ell == pytest.approx([0.9, 1.35, 1.35, 0.9])  # all above G_thres -> f_small
    assert keep.tolist() == [1, 1, 1, 1]  # f_small < 1 keeps everything
    Gf, L, ell, keep = orc.reduce(pos, off, nbr, f, 0.9, 2.1, 0.75, seed=1)
    assert ell == pytest.approx([2.1, 2.1 * 1.5, 1.35, 0.9])


def test_zero_tracer_pair_and_isolated_point(orc):
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [5.0, 5.0, 5.0]])
    off = np.array([0, 1, 2, 2])
    nbr = np.array([1, 0], np.int32)
    Gf, L, ell, keep = orc.reduce(pos, off, nbr, np.zeros(3), 1.0, 2.15, 0.21, seed=3)
    assert Gf.tolist() == [0.0, 0.0, 0.0]
    assert L.tolist() == [1.0, 1.0, 0.0]
    assert keep[2] == 1  # no neighbours: kept


def test_range_and_thinning_rate(orc):
    import synth

    m = synth.wind_model(3000, seed=5)
    f = m["rho"] * np.exp(np.random.default_rng(0).normal(0, 0.3, 3000))
    Gf, L, ell, keep = orc.reduce(m["pos"], m["nbr_off"], m["nbr_idx"], f, 1.0, 2.15, 0.21, seed=9)
    assert Gf.min() >= 0.0 and Gf.max() <= 1.0
    small = Gf >= 0.21
    assert keep[small].all()  # f_small = 1: p = 1
    p = 1 / 2.15 ** 3
    n = (~small).sum()
    k = keep[~small].sum()
    sd = math.sqrt(n * p * (1 - p))
    assert abs(k - n * p) < 5 * sd
