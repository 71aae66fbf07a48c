"""Learned surrogate of the dominant NPF magnitudes over a family of operating points.

Not part of the paper's method: the paper computes NPFs per operating point (Section II,
Algorithm 2). Here a small MLP ensemble, trained on NPFs from the plain method, maps an
operating-point parameter vector p to |NPF| at a fixed set of (state, mode) entries; the plain
method stays the reference and the fallback for every query on which the ensemble members
disagree by more than a relative spread limit.

Pipeline of one query p: A1(p) -> eigen-triple (host LAPACK; the method's input) -> either the
surrogate (one forward pass of every member, npf_mlp_predict) or, when gated, the plain GPU method
(npf_set_modes + npf_batch_compute) -> |NPF| at the index set.
"""
from __future__ import annotations

import numpy as np

from . import OPT_TILE_N, Plan, batch_compute
from .mlp import Mlp, param_layout


def modal_data(A, lam_ref=None):
    """Eigen-triple (lam, U, V = U^-1) of a real matrix. With lam_ref the modes are reordered to
    match it (minimum total |lam - lam_ref| assignment), so that mode i keeps its identity over a
    family of operating points."""
    lam, U = np.linalg.eig(np.asarray(A, dtype=np.float64))
    if lam_ref is not None:
        from scipy.optimize import linear_sum_assignment
        cost = np.abs(lam[:, None] - np.asarray(lam_ref)[None, :])
        r, c = linear_sum_assignment(cost)
        order = np.empty_like(r)
        order[c] = r
        lam, U = lam[order], U[:, order]
    V = np.linalg.inv(U)
    return lam.astype(np.complex128), U.astype(np.complex128), V.astype(np.complex128)


def top_indices(npf, k=64):
    """Flat indices (k * n + i) of the k largest |NPF[k, i]|; equal magnitudes go to the lower
    flat index."""
    a = np.abs(np.asarray(npf)).ravel()
    return np.argsort(-a, kind="stable")[:k]


class PlainSolver:
    """|NPF| at fixed entries for many operating points of one family, by the plain method: a
    pool of plans whose modal data are replaced per query, computed in batches through one
    recorded graph per pool size."""

    def __init__(self, fam, order, lam_ref, indices=None, slots=256, precision="split_bf16"):
        self.fam = fam
        self.order = order
        self.lam_ref = np.asarray(lam_ref)
        self.indices = None if indices is None else np.asarray(indices)
        lam, U, V = modal_data(fam.A(fam.p0), self.lam_ref)
        self.plans = []
        for _ in range(slots):
            p = Plan(lam, U, V, order, precision=precision)
            p.set_option(OPT_TILE_N, 0)   # tile width autotuned
            for N, t in fam.tensors.items():
                if N <= order:
                    p.set_tensor(N, t)
            self.plans.append(p)
        n = fam.n
        self.outs = [np.empty((n, n), np.complex128) for _ in range(slots)]

    def npf(self, P):
        """Full NPF matrices [len(P), n, n]."""
        P = np.atleast_2d(P)
        res = np.empty((len(P), self.fam.n, self.fam.n), np.complex128)
        S = len(self.plans)
        for c0 in range(0, len(P), S):
            m = min(S, len(P) - c0)
            for j in range(m):
                self.plans[j].set_modes(*modal_data(self.fam.A(P[c0 + j]), self.lam_ref))
            batch_compute(self.plans[:m], [self.order] * m, self.outs[:m])
            for j in range(m):
                res[c0 + j] = self.outs[j]
        return res

    def values(self, P):
        """|NPF| at the index set, [len(P), k]."""
        F = self.npf(P)
        return np.abs(F.reshape(len(F), -1)[:, self.indices])

    def close(self):
        for p in self.plans:
            p.close()
        self.plans = []


def init_weights(widths, ensemble, seed=0):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases; member e from seed + e."""
    out = []
    for e in range(ensemble):
        rng = np.random.default_rng(seed + e)
        parts = []
        for (r, c) in param_layout(widths):
            W = np.zeros((r, c), np.float32)
            b = np.sqrt(6.0 / (c - 1))
            W[:, :-1] = rng.uniform(-b, b, (r, c - 1))
            parts.append(W.ravel())
        out.append(np.concatenate(parts))
    return np.stack(out)


class Surrogate:
    """MLP ensemble on standardised log|NPF| at a fixed index set."""

    def __init__(self, fam, indices, widths, ensemble=5, seed=0):
        self.fam = fam
        self.indices = np.asarray(indices)
        self.widths = list(widths)
        self.net = Mlp(widths, init_weights(widths, ensemble, seed))
        self.mu = np.zeros(widths[-1], np.float32)
        self.sigma = np.ones(widths[-1], np.float32)

    def features(self, P):
        P = np.atleast_2d(np.asarray(P, dtype=np.float64))
        return (2.0 * (P - self.fam.lo) / (self.fam.hi - self.fam.lo) - 1.0).astype(np.float32)

    def fit(self, P, values, epochs=300, batch=256, lr=1e-3, seed=0):
        """Train every member on |NPF| values [len(P), k]; returns the per-epoch loss."""
        t = np.log(np.asarray(values, dtype=np.float64))
        self.mu = t.mean(axis=0).astype(np.float32)
        self.sigma = np.maximum(t.std(axis=0), 1e-6).astype(np.float32)
        T = ((t - self.mu) / self.sigma).astype(np.float32)
        return self.net.train(self.features(P), T, epochs, batch, lr, seed)

    def predict(self, P, spread_limit=0.05):
        """Ensemble mean |NPF| [len(P), k], largest relative spread [len(P)], fallback mask."""
        return self.net.predict(self.features(P), self.mu, self.sigma, spread_limit)

    def gated(self, P, solver, spread_limit=0.05):
        """Surrogate values where the members agree, the plain method's elsewhere."""
        mean, spread, fb = self.predict(P, spread_limit)
        out = mean.astype(np.float64)
        if fb.any():
            out[fb] = solver.values(np.atleast_2d(P)[fb])
        return out, spread, fb

    def close(self):
        self.net.close()
