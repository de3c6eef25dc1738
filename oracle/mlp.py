"""Plain FP64 NumPy oracle of the learned mesh-reduction network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the CUDA training and
inference kernels are checked against this file; they never call it.

Network (8 -> 64 -> 64 -> 1, ReLU), parameters in one flat vector theta:
    W1 [8][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]
    h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 . W3 + b3
Loss: mean squared error over the batch, L = mean_i (y_i - t_i)^2.

With bf16=True the values that the GPU kernels hold in bfloat16 (the inputs,
W1, W2, the activations h1, and the output gradients of the second and first
layers) are rounded to bfloat16 (round to nearest even) at the same places,
and everything else is computed in double precision, so that the comparison
isolates the kernels' single-precision accumulation.
"""
from __future__ import annotations

import numpy as np

SHAPES = (("W1", (8, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64,)), ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[k:k + size].reshape(shape)
        k += size
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, bf=False):
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    W1, W2 = p["W1"], p["W2"]
    if bf:
        X, W1, W2 = bf16(X), bf16(W1), bf16(W2)
    a1 = X @ W1 + p["b1"]
    h1 = np.maximum(a1, 0.0)
    if bf:
        h1 = bf16(h1)
    a2 = h1 @ W2 + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, dict(X=X, W1=W1, W2=W2, h1=h1, h2=h2)


def loss_and_grad(theta, X, t, bf=False):
    """MSE loss and its gradient with respect to theta (manual backward)."""
    p = unpack(theta)
    y, c = forward(theta, X, bf)
    t = np.asarray(t, np.float64)
    n = len(t)
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["b3"] = np.array([dy.sum()])
    g["W3"] = c["h2"].T @ dy
    dh2 = np.outer(dy, p["W3"]) * (c["h2"] > 0)
    if bf:
        dh2 = bf16(dh2)
    g["b2"] = dh2.sum(0)
    g["W2"] = c["h1"].T @ dh2
    dh1 = (dh2 @ c["W2"].T) * (c["h1"] > 0)
    if bf:
        dh1 = bf16(dh1)
    g["b1"] = dh1.sum(0)
    g["W1"] = c["X"].T @ dh1
    return L, pack(g)


def grad_magnitudes(theta, X, t, bf=False):
    """For every gradient element, the sum of the magnitudes of the terms that
    loss_and_grad adds up for it (|h|^T |d| for a weight, sum |d| for a bias):
    the scale against which the rounding of a differently ordered or
    differently rounded evaluation of the same sums is measured."""
    p = unpack(theta)
    y, c = forward(theta, X, bf)
    t = np.asarray(t, np.float64)
    n = len(t)
    ady = np.abs(2.0 * (y - t) / n)
    g = {}
    g["b3"] = np.array([ady.sum()])
    g["W3"] = np.abs(c["h2"]).T @ ady
    adh2 = np.outer(ady, np.abs(p["W3"])) * (c["h2"] > 0)
    g["b2"] = adh2.sum(0)
    g["W2"] = np.abs(c["h1"]).T @ adh2
    adh1 = (adh2 @ np.abs(c["W2"]).T) * (c["h1"] > 0)
    g["b1"] = adh1.sum(0)
    g["W1"] = np.abs(c["X"]).T @ adh1
    return pack(g)


def init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = dict(W1=rng.normal(0, np.sqrt(2 / 8), (8, 64)), b1=np.zeros(64),
             W2=rng.normal(0, np.sqrt(2 / 64), (64, 64)), b2=np.zeros(64),
             W3=rng.normal(0, np.sqrt(1 / 64), 64), b3=np.zeros(1))
    return pack(p)


def features(pos, vel, nbr_off, nbr_idx, rho, T, dvw, chi0_line0):
    """Eight per-point features of the reduction network (plain loops of NumPy
    rows): log rho, max |log rho_n - log rho_i|, max |v_n - v_i| / dv_i, log T,
    log L_i (mean neighbour distance, Eq. 8), degree, log |x_i|,
    log (chi0_i L_i)."""
    n = len(pos)
    X = np.zeros((n, 8))
    lr = np.log(np.asarray(rho, np.float64))
    for i in range(n):
        nb = np.asarray(nbr_idx[nbr_off[i]:nbr_off[i + 1]], np.int64)
        d = np.sqrt(((pos[nb] - pos[i]) ** 2).sum(1)) if len(nb) else np.zeros(0)
        L = d.mean() if len(nb) else 0.0
        X[i, 0] = lr[i]
        X[i, 1] = np.abs(lr[nb] - lr[i]).max() if len(nb) else 0.0
        X[i, 2] = (np.sqrt(((vel[nb] - vel[i]) ** 2).sum(1)).max() if len(nb) else 0.0) / dvw[i]
        X[i, 3] = np.log(T[i])
        X[i, 4] = np.log(L + 1e-30)
        X[i, 5] = len(nb)
        X[i, 6] = np.log(np.sqrt((pos[i] ** 2).sum()) + 1e-30)
        X[i, 7] = np.log(chi0_line0[i] * L + 1e-30)
    return X
