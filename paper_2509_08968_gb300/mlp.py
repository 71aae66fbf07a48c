"""Binding of the surrogate MLP ensemble (include/npf_mlp.h): argument marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import NpfError, _check, _ptr, load


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def param_layout(widths):
    """[(out, in + 1)] per layer: the public weight layout, bias in the last column."""
    return [(widths[l + 1], widths[l] + 1) for l in range(len(widths) - 1)]


def unflatten(flat, widths):
    """One member's flat weight vector -> list of [out, in + 1] matrices."""
    mats, o = [], 0
    for r, c in param_layout(widths):
        mats.append(flat[o:o + r * c].reshape(r, c))
        o += r * c
    return mats


class Mlp:
    """An ensemble of `weights.shape[0]` members with layer widths `widths` (inputs first)."""

    def __init__(self, widths, weights, stream=None):
        lib = load()
        self.widths = [int(w) for w in widths]
        self.L = len(self.widths) - 1
        weights = _f32(weights)
        self.E = int(weights.shape[0])
        wd = (ctypes.c_int * len(self.widths))(*self.widths)
        h = lib.npf_mlp_create(self.E, self.L, wd, _ptr(weights),
                               ctypes.c_void_p(stream or 0))
        if not h:
            raise NpfError(lib.npf_last_status(), lib.npf_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)
        self.params = int(lib.npf_mlp_param_count(self._h))

    def weights(self):
        out = np.empty((self.E, self.params), np.float32)
        _check(load().npf_mlp_get_weights(self._h, _ptr(out)))
        return out

    def forward(self, X):
        X = _f32(X)
        Y = np.empty((self.E, X.shape[0], self.widths[-1]), np.float32)
        _check(load().npf_mlp_forward(self._h, X.shape[0], _ptr(X), _ptr(Y)))
        return Y

    def loss_grad(self, X, T):
        X, T = _f32(X), _f32(T)
        g = np.empty((self.E, self.params), np.float32)
        loss = np.empty(self.E, np.float32)
        _check(load().npf_mlp_loss_grad(self._h, X.shape[0], _ptr(X), _ptr(T), _ptr(g),
                                        _ptr(loss)))
        return loss, g

    def train(self, X, T, epochs, batch, lr, seed=0):
        X, T = _f32(X), _f32(T)
        hist = np.empty(max(epochs, 1), np.float32)
        _check(load().npf_mlp_train(self._h, X.shape[0], _ptr(X), _ptr(T), int(epochs),
                                    int(batch), float(lr), ctypes.c_uint64(seed), _ptr(hist)))
        return hist[:epochs]

    def predict(self, X, mu, sigma, spread_limit=0.05):
        X = _f32(X)
        R, wo = X.shape[0], self.widths[-1]
        mean = np.empty((R, wo), np.float32)
        spread = np.empty(R, np.float32)
        fb = np.empty(R, np.int32)
        _check(load().npf_mlp_predict(self._h, R, _ptr(X), _ptr(_f32(mu)), _ptr(_f32(sigma)),
                                      float(spread_limit), _ptr(mean), _ptr(spread), _ptr(fb)))
        return mean, spread, fb.astype(bool)

    def close(self):
        if getattr(self, "_h", None):
            load().npf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
