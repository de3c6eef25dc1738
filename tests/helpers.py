"""Shared test helpers (comparison metrics); no method arithmetic."""
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
