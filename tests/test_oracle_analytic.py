"""Pins of the oracle's element-size field for analytic models (Section 2.2.1,
Eq. 5: Gf = ||grad f|| / f on a Cartesian background mesh, mapped linearly
from [max Gf, min Gf] onto [ell_min, ell_max]) and of its thinning.

* An exponential tracer along one axis has the closed-form central difference
  Gf = sinh(a h) / h inside and (e^{ah} - 1)/h, (1 - e^{-ah})/h on the faces.
* A Gaussian tracer approaches Gf = r / sigma^2 at second order in h.
* ell is affine in Gf with the stated endpoints; a constant tracer gives ell_max.
* The kept fraction follows (h / ell)^3 in distribution.
"""
import math

import numpy as np


def test_exponential_closed_form(orc):
    a, h, nx = 0.7, 0.3, 11
    x = np.arange(nx) * h
    f = np.repeat(np.exp(a * x)[:, None, None], 3, axis=1)  # [nx, 3, 1]
    Gf, ell, keep = orc.analytic_mesh(f, h, h, 4 * h, seed=1)
    assert np.allclose(Gf[1:-1], math.sinh(a * h) / h, rtol=1e-13)
    assert np.allclose(Gf[0], (math.exp(a * h) - 1) / h, rtol=1e-13)
    assert np.allclose(Gf[-1], (1 - math.exp(-a * h)) / h, rtol=1e-13)


def _gauss(n, sigma=0.2):
    h = 1.0 / (n - 1)
    g = np.arange(n) * h - 0.5
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt(X**2 + Y**2 + Z**2)
    return np.exp(-r**2 / (2 * sigma**2)), r, h, sigma


def test_gaussian_converges_at_second_order(orc):
    errs = []
    for n in (17, 33, 65):
        f, r, h, s = _gauss(n)
        Gf, _, _ = orc.analytic_mesh(f, h, h, 0.25, seed=2)
        inner = (slice(1, -1),) * 3
        errs.append(np.median(np.abs(Gf[inner] - r[inner] / s**2)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_linear_map_and_constant_tracer(orc):
    f, r, h, s = _gauss(17)
    emin, emax = h, 0.25
    Gf, ell, keep = orc.analytic_mesh(f, h, emin, emax, seed=3)
    assert ell.flat[np.argmax(Gf)] == emin and ell.flat[np.argmin(Gf)] == emax
    coef = np.polyfit(Gf.ravel(), ell.ravel(), 1)
    assert np.allclose(np.polyval(coef, Gf.ravel()), ell.ravel(), rtol=0, atol=1e-12)
    assert coef[0] < 0
    Gc, ellc, keepc = orc.analytic_mesh(np.full((5, 4, 3), 2.0), 0.1, 0.1, 0.4, seed=4)
    assert np.all(Gc == 0.0) and np.all(ellc == 0.4)


def test_thinning_rate(orc):
    f, r, h, s = _gauss(41)
    Gf, ell, keep = orc.analytic_mesh(f, h, 1.5 * h, 0.2, seed=5)
    assert ell.min() == 1.5 * h
    p = (h / ell.ravel()) ** 3
    k = keep.sum()
    assert abs(k - p.sum()) < 5 * math.sqrt((p * (1 - p)).sum())
    # the densest region is around the Gaussian's inflection shell r = sigma, not the centre
    assert keep[np.abs(r - s) < 0.05].mean() > 3 * keep[r < 0.05].mean()
