"""Mesh reduction workflow around the CUDA kernels (Section 2.2.2).

The reduction criterion (Eqs. 6-8) and the learned network run in libmgx;
this module does the host-side parts of the workflow that the paper leaves to
other tools: re-meshing a thinned point set (a Delaunay tetrahedralisation
of the kept points, in place of Gmsh), mapping J of a reduced mesh back to the
full one by barycentric interpolation (as the paper does with SciPy's
LinearNDInterpolator, Section 3.2.1), the per-point relative error, and the
data set that trains the reduction network: for points that plain reductions
dropped, the log10 of the J error their absence caused.
"""
from __future__ import annotations

import numpy as np

from . import (MGX_FP32, mgx_mlp_features, mgx_mlp_get_params, mgx_mlp_set_params, mgx_mlp_train,
               mgx_reduce_mesh_learned, mgx_reduce_mesh_learned_weighted)

POINT_FIELDS = ("pos", "vel", "chi0", "eta0", "dvw", "chi_c", "eta_c", "rho", "T")


def delaunay_neighbours(pos: np.ndarray):
    """CSR neighbour lists (sorted, symmetric) from the Delaunay edges."""
    from scipy.spatial import Delaunay

    n = len(pos)
    s = Delaunay(pos).simplices.astype(np.int64)
    a = np.concatenate([s[:, i] for i in range(4) for j in range(i + 1, 4)])
    b = np.concatenate([s[:, j] for i in range(4) for j in range(i + 1, 4)])
    src, dst = np.concatenate([a, b]), np.concatenate([b, a])
    key = np.unique(src * n + dst)
    src, dst = key // n, key % n
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    return np.cumsum(off), dst.astype(np.int32)


def remesh(m: dict, keep: np.ndarray) -> dict:
    """The model restricted to the kept points, with fresh Delaunay neighbours."""
    idx = np.where(np.asarray(keep) != 0)[0]
    out = dict(m)
    for k in POINT_FIELDS:
        if k in m:
            out[k] = np.ascontiguousarray(np.asarray(m[k])[idx])
    out["nbr_off"], out["nbr_idx"] = delaunay_neighbours(out["pos"])
    out["sample"] = np.arange(min(len(idx), 10000), dtype=np.int32)
    out["name"] = m.get("name", "model") + f"_reduced{len(idx)}"
    return out


def interpolate(pos_src: np.ndarray, values: np.ndarray, pos_dst: np.ndarray) -> np.ndarray:
    """Barycentric (linear) interpolation on the Delaunay mesh of pos_src, with
    the nearest source point outside its convex hull."""
    from scipy.interpolate import LinearNDInterpolator
    from scipy.spatial import cKDTree

    lin = LinearNDInterpolator(pos_src, values)(pos_dst)
    bad = ~np.isfinite(lin).all(axis=1)
    if bad.any():
        _, nn = cKDTree(pos_src).query(pos_dst[bad])
        lin[bad] = values[nn]
    return lin


def point_errors(J_full: np.ndarray, J_approx: np.ndarray, floor: float = 1e-6) -> np.ndarray:
    """Relative error per point, averaged over the bins where J exceeds `floor`
    times the point's maximum (the paper averages over directions and bins)."""
    mask = J_full > floor * J_full.max(axis=1, keepdims=True)
    rel = np.where(mask, np.abs(J_approx - J_full) / np.where(mask, J_full, 1.0), 0.0)
    return rel.sum(1) / np.maximum(mask.sum(1), 1)


def reduction_error(ctx, m: dict, J_full: np.ndarray, keep: np.ndarray, precision: int = MGX_FP32, **solve):
    """Per-point error of J after reducing m to the kept points."""
    r = remesh(m, keep)
    mid = ctx.load(r)
    try:
        J_red = ctx.solve_J(mid, precision=precision, **solve)
    finally:
        ctx.free(mid)
    return point_errors(J_full, interpolate(r["pos"], J_red, m["pos"]))


class Standardizer:
    def __init__(self, X: np.ndarray):
        self.mean = X.mean(0)
        self.std = np.maximum(X.std(0), 1e-6)

    def __call__(self, X: np.ndarray) -> np.ndarray:
        return ((X - self.mean) / self.std).astype(np.float32)


def training_samples(ctx, m: dict, reductions, label_floor: float = 1e-4, **solve):
    """Features of the points that each plain reduction (f_small, f_large,
    G_thres, seed) drops, and the log10 of their J error after re-meshing."""
    mid = ctx.load(m)
    try:
        J_full = ctx.solve_J(mid, precision=MGX_FP32, **solve)
        X = mgx_mlp_features(ctx.ptr, mid, m["rho"], m["T"])
        Xs, ys = [], []
        for f_small, f_large, g_thres, seed in reductions:
            keep = ctx.reduce_mesh(mid, m["rho"], f_small, f_large, g_thres, seed)[3]
            err = reduction_error(ctx, m, J_full, keep, **solve)
            drop = keep == 0
            Xs.append(X[drop])
            ys.append(np.log10(err[drop] + label_floor))
    finally:
        ctx.free(mid)
    return np.concatenate(Xs), np.concatenate(ys).astype(np.float32)


def train_network(ctx, X: np.ndarray, y: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 2e-3,
                  seed: int = 0):
    """Standardise the features, initialise (He-normal) and train on the GPU."""
    std = Standardizer(X)
    rng = np.random.default_rng(seed)
    theta = np.concatenate([rng.normal(0, np.sqrt(2 / 8), 512), np.zeros(64), rng.normal(0, np.sqrt(2 / 64), 4096),
                            np.zeros(64), rng.normal(0, np.sqrt(1 / 64), 64), [float(y.mean())]])
    mgx_mlp_set_params(ctx.ptr, theta.astype(np.float32))
    losses = mgx_mlp_train(ctx.ptr, std(X), y, epochs, batch, lr, seed)
    return std, losses, mgx_mlp_get_params(ctx.ptr)


def reduce_learned(ctx, mid: int, m: dict, std: Standardizer, keep_fraction: float) -> np.ndarray:
    """Keep the points whose predicted J error (if dropped) is largest."""
    X = mgx_mlp_features(ctx.ptr, mid, m["rho"], m["T"])
    keep, _ = mgx_reduce_mesh_learned(ctx.ptr, mid, std(X), keep_fraction)
    return keep


def reduce_learned_weighted(ctx, mid: int, m: dict, std: Standardizer, keep_fraction: float, alpha: float = 2.0,
                            seed: int = 0) -> np.ndarray:
    """Keep each point with probability min(1, c 10^(alpha y)), y its predicted
    log10 J error if dropped, c matching the expected count to keep_fraction."""
    X = mgx_mlp_features(ctx.ptr, mid, m["rho"], m["T"])
    keep, _, _ = mgx_reduce_mesh_learned_weighted(ctx.ptr, mid, std(X), keep_fraction, alpha, seed)
    return keep
