"""Shared test helpers (comparison metrics, tiny hand-built models); no method arithmetic."""
import numpy as np


def j_rel_err(Jg, Jo, floor=1e-6):
    """Largest relative error of J over the bins where the reference exceeds
    `floor` times its maximum over the bins of that point, and the largest
    absolute error over all bins."""
    Jg = np.asarray(Jg, np.float64)
    Jo = np.asarray(Jo, np.float64)
    mx = np.abs(Jo).max(axis=1, keepdims=True)
    mask = np.abs(Jo) > floor * mx
    rel = np.abs(Jg - Jo)[mask] / np.abs(Jo[mask]) if mask.any() else np.zeros(1)
    return float(rel.max()), float(np.abs(Jg - Jo).max())


def line_model(vel_a, vel_b, dv=1.0):
    """Three points on the x axis (0, 1, 2), chained neighbours, origin in the middle."""
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    off = np.array([0, 1, 3, 4])
    nbr = np.array([1, 0, 2, 1], np.int32)
    vel = np.array([[vel_a, 0, 0], [0.0, 0, 0], [vel_b, 0, 0]])
    one = np.ones((3, 1))
    return dict(pos=pos, vel=vel, nbr_off=off, nbr_idx=nbr, nu0=np.array([1e11]), chi0=one,
                eta0=one, dvw=np.full(3, dv), chi_c=np.full(3, 1e-3), eta_c=np.full(3, 1e-3),
                n_freq=3, x_span=2.0, l_min=0, l_max=0)


def oracle_model_of(orc, pos, off, nbr):
    """An oracle model of a bare mesh (one static line of unit data, no ray set),
    for tracing only."""
    n = len(pos)
    m = dict(pos=pos, vel=np.zeros((n, 3)), nbr_off=off, nbr_idx=nbr, nu0=np.array([1.0]), chi0=np.ones((n, 1)),
             eta0=np.ones((n, 1)), dvw=np.ones(n), chi_c=np.ones(n), eta_c=np.ones(n), n_freq=1, x_span=0.0,
             l_min=0, l_max=0)
    return orc.OracleModel(m, rays=np.zeros((n, 6), np.uint32))
