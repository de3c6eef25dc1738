"""Meshing of analytic models (Section 2.2.1) around the CUDA size-field kernel.

The element-size field (Eq. 5) and the thinning of the background mesh run in
libmgx (`mgx_analytic_mesh`); this module lays out the regular Cartesian
background mesh, evaluates the caller's tracer function on it, offsets the kept
points by a seeded sub-cell jitter (a regular lattice has degenerate Delaunay
simplices) and connects them by a Delaunay tetrahedralisation, in place of Gmsh.
"""
from __future__ import annotations

import numpy as np

from . import mgx_analytic_mesh
from .learned import delaunay_neighbours


def background_grid(lo, hi, h):
    """Axes of the regular background mesh of spacing h covering [lo, hi]^3 (per axis)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n = np.floor((hi - lo) / h + 1e-9).astype(int) + 1
    return [lo[a] + h * np.arange(n[a]) for a in range(3)]


def analytic_mesh(ctx, tracer, lo, hi, h, ell_min, ell_max, seed=0, jitter=0.25):
    """Mesh of an analytic model: tracer(x [..., 3]) > 0 evaluated on the
    background mesh of spacing h over [lo, hi]^3, its element-size field and
    thinning on the GPU, the kept points jittered by up to jitter * h per axis
    and joined by Delaunay.  Returns dict(pos, nbr_off, nbr_idx, Gf, ell, keep,
    shape, h)."""
    axes = background_grid(lo, hi, h)
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([X, Y, Z], axis=-1)
    f = np.ascontiguousarray(tracer(pts), np.float64)
    Gf, ell, keep, n_kept = mgx_analytic_mesh(ctx.ptr, f, h, ell_min, ell_max, seed)
    pos = pts.reshape(-1, 3)[keep.ravel() != 0]
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x1E]))
    pos = pos + rng.uniform(-jitter * h, jitter * h, pos.shape)
    off, nbr = delaunay_neighbours(pos)
    return dict(pos=pos, nbr_off=off, nbr_idx=nbr, Gf=Gf, ell=ell, keep=keep, shape=f.shape, h=h, n_kept=n_kept)
