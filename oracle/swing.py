"""Packed derivative tensors of the swing model (npf_synth.SwingModel), CPU oracle (test
infrastructure only: tests/, the package smoke check and the benchmark's CPU-baseline leg may
import it; the library never does).

A_N[e, q] = d^N f_e / dx_{s_0} .. dx_{s_{N-1}} at the equilibrium for the q-th non-decreasing
tuple s of state indices. Only the network terms of the omega equations depend on x beyond first
order, and only through the angle differences t_jk = delta_j - delta_k (and delta_j itself for a
line to the reference bus): with a derivatives in delta_j and b in delta_k (a + b = N) a line
contributes (-1)^b d^N/dt^N [G_jk cos t + B_jk sin t], each N-th derivative of cos / sin being a
quarter-turn phase shift.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _gN(G, B, t, N):
    return G * math.cos(t + N * math.pi / 2) + B * math.sin(t + N * math.pi / 2)


def packed_tensor(model, N):
    """[2m, C(2m+N-1, N)] float64."""
    m = model.m
    n = 2 * m
    tuples = list(itertools.combinations_with_replacement(range(n), N))
    A = np.zeros((n, len(tuples)))
    for q, s in enumerate(tuples):
        if max(s) >= m:
            continue
        vals = sorted(set(s))
        if len(vals) > 2:
            continue
        for j in range(m):
            coef = -model.V[j] / (2.0 * model.H[j])
            total = 0.0
            for k in range(m):
                if k == j:
                    continue
                a = s.count(j)
                b = s.count(k)
                if a + b != N:
                    continue
                total += (-1) ** b * model.V[k] * _gN(model.G[j, k], model.B[j, k],
                                                      model.delta[j] - model.delta[k], N)
            if s.count(j) == N:   # line to the reference bus (voltage 1, angle 0)
                total += _gN(model.Gb[j], model.Bb[j], model.delta[j], N)
            A[m + j, q] = coef * total
    return A


def finite_difference_tensor(model, N, h=1e-3):
    """Central-difference estimate of the packed order-N tensor from f alone (step h; error
    O(h^2) plus rounding O(eps / h^N))."""
    m = model.m
    n = 2 * m
    x0 = np.concatenate([model.delta, np.zeros(m)])
    tuples = list(itertools.combinations_with_replacement(range(n), N))
    A = np.zeros((n, len(tuples)))
    for q, s in enumerate(tuples):
        acc = np.zeros(n)
        for signs in itertools.product((1, -1), repeat=N):
            x = x0.copy()
            for idx, sg in zip(s, signs):
                x[idx] += sg * h
            acc += np.prod(signs) * model.f(x)
        A[:, q] = acc / (2 * h) ** N
    return A
