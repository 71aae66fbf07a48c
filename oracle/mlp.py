"""CPU oracle of the surrogate network (test infrastructure only: tests/, the package smoke check
and the benchmark's CPU-baseline leg may import it; the library never does).

Plain NumPy float64 forward pass, mean-squared-error loss and back-propagation of a multilayer
perceptron

    z_l = W_l h_l + b_l,   h_{l+1} = relu(z_l) (l < L-1),   y = z_{L-1},
    loss = (1 / (R w_L)) sum_{r,o} (y_ro - t_ro)^2,

with the weights in the library's public layout: per layer a matrix [w_{l+1}][w_l + 1] whose last
column is the bias. With bf16=True every value that enters a product in the GPU kernels (the
inputs, the weights and biases, the hidden activations, the output error and the back-propagated
errors) is first rounded to bfloat16 (round to nearest, ties to even), so that the two sides take
the same rounding decisions; the sums stay float64.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64. bfloat16 keeps the top
    16 bits of an IEEE binary32: the value is first rounded to binary32, then the low 16 bits are
    rounded away."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(x, bf16):
    return round_bf16(x) if bf16 else np.asarray(x, dtype=np.float64)


def forward(mats, X, bf16=False):
    """Outputs y [R, w_L] and the per-layer inputs h_l [R, w_l] (as used in the products)."""
    h = _q(X, bf16)
    hs = []
    for l, M in enumerate(mats):
        M = _q(M, bf16)
        W, b = M[:, :-1], M[:, -1]
        hs.append(h)
        z = h @ W.T + b
        if l + 1 < len(mats):
            h = _q(np.maximum(z, 0.0), bf16)
        else:
            return z, hs
    raise ValueError("no layers")


def loss_grad(mats, X, T, bf16=False):
    """Mean-squared-error loss and its gradient with respect to every [W_l | b_l]."""
    y, hs = forward(mats, X, bf16)
    T = np.asarray(T, dtype=np.float64)
    R, wo = y.shape
    d = y - T
    loss = float((d * d).sum() / (R * wo))
    dz = _q(2.0 * d / (R * wo), bf16)
    grads = [None] * len(mats)
    for l in range(len(mats) - 1, -1, -1):
        h = hs[l]
        ha = np.concatenate([h, np.ones((R, 1))], axis=1)
        grads[l] = dz.T @ ha
        if l == 0:
            break
        W = _q(mats[l], bf16)[:, :-1]
        dz = _q((dz @ W) * (h > 0.0), bf16)
    return loss, grads
