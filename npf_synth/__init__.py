"""Seeded synthetic inputs for the NPF computation.

This module only builds inputs: a diagonalisable state matrix with its eigen-triple
(lambda, U = right eigenvectors Phi, V = U^-1 = left eigenvectors Psi) and real Taylor
coefficient tensors A_N that are symmetric in their N lower indices. It holds none of the
method's arithmetic (no mode products, no resonance divide, no NPF reduction), so both the
CUDA path and the CPU oracle may draw from it.

Packed layout of a symmetric tensor (the library's input format):
    coeffs[j, r] = A_N^j_{a_1 .. a_N} for the r-th non-decreasing tuple a_1 <= .. <= a_N in
    lexicographic order, i.e. the order of itertools.combinations_with_replacement(range(n), N).
    Shape [n, C(n+N-1, N)], float64, upper index j outermost.

Eigen-structure recipe (the paper's models are not available; these stand in for their sizes):
    A_1 = P . blockdiag(B_b) . P^-1 with B_b = [[s, w], [-w, s]], s ~ U[-2, -0.05], w ~ U[0.5, 15]
    rad/s, so each block carries the complex-conjugate mode pair s +- i w with eigenvectors
    [1, +-i]. Then U = P . blockdiag([[1, 1], [i, -i]]) and V = U^-1 exactly.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

SIGMA_RANGE = (-2.0, -0.05)
OMEGA_RANGE = (0.5, 15.0)


def packed_count(n: int, N: int) -> int:
    """Number of non-decreasing N-tuples over range(n): C(n+N-1, N)."""
    return math.comb(n + N - 1, N)


def sorted_tuples(n: int, N: int):
    """All non-decreasing N-tuples over range(n) in packed (lexicographic) order."""
    return itertools.combinations_with_replacement(range(n), N)


@dataclass
class ModalSystem:
    n: int
    A1: np.ndarray          # real [n, n]
    lam: np.ndarray         # complex [n]
    U: np.ndarray           # complex [n, n], column p = right eigenvector (phi_{a p} = U[a, p])
    V: np.ndarray           # complex [n, n], row i = left eigenvector (psi_{i k} = V[i, k])
    P: np.ndarray           # real [n, n] similarity used to build A1
    tensors: dict = field(default_factory=dict)   # order N -> packed float64 [n, C(n+N-1, N)]


def _block_pair_eigvecs(nblk2: int) -> np.ndarray:
    """blockdiag([[1, 1], [i, -i]]) for nblk2 2x2 blocks."""
    W = np.zeros((2 * nblk2, 2 * nblk2), dtype=np.complex128)
    for b in range(nblk2):
        W[2 * b, 2 * b] = 1.0
        W[2 * b, 2 * b + 1] = 1.0
        W[2 * b + 1, 2 * b] = 1.0j
        W[2 * b + 1, 2 * b + 1] = -1.0j
    return W


def _cond(M: np.ndarray) -> float:
    s = np.linalg.svd(M, compute_uv=False)
    return float(s[0] / s[-1])


def modal_system(n: int, seed: int, block: int = 2, coupling: float = 0.0,
                 coupling_density: float = 0.10, p_scale: float = 0.3,
                 cond_max: float = 1e3, sigmas=None, omegas=None) -> ModalSystem:
    """Diagonalisable real A1 with known eigen-triple.

    block=2: P = I + p_scale * N(0,1) (dense), rejected until cond(P) < cond_max.
    block=4: P block-diagonal with 4x4 blocks I + p_scale*N(0,1) (each cond < cond_max), plus a
             fraction `coupling_density` of off-block entries set to N(0, coupling), the whole P
             again checked against cond_max ("generator-like blocks with sparse inter-block
             coupling").
    """
    if n % 2:
        raise ValueError("n must be even (modes come in complex-conjugate pairs)")
    rng = np.random.default_rng(seed)
    npairs = n // 2
    s = rng.uniform(*SIGMA_RANGE, size=npairs) if sigmas is None else np.asarray(sigmas, float)
    w = rng.uniform(*OMEGA_RANGE, size=npairs) if omegas is None else np.asarray(omegas, float)
    B = np.zeros((n, n))
    for b in range(npairs):
        B[2 * b:2 * b + 2, 2 * b:2 * b + 2] = [[s[b], w[b]], [-w[b], s[b]]]
    for _attempt in range(1000):
        if block == 2:
            P = np.eye(n) + p_scale * rng.standard_normal((n, n))
        elif block == 4:
            if n % 4:
                raise ValueError("block=4 needs n % 4 == 0")
            P = np.zeros((n, n))
            for b in range(n // 4):
                while True:
                    Pb = np.eye(4) + p_scale * rng.standard_normal((4, 4))
                    if _cond(Pb) < cond_max:
                        break
                P[4 * b:4 * b + 4, 4 * b:4 * b + 4] = Pb
            if coupling > 0.0:
                blk = np.arange(n) // 4
                off = blk[:, None] != blk[None, :]
                mask = off & (rng.random((n, n)) < coupling_density)
                P[mask] = coupling * rng.standard_normal(int(mask.sum()))
        else:
            raise ValueError("block must be 2 or 4")
        if _cond(P) < cond_max:
            break
    else:  # pragma: no cover
        raise RuntimeError("could not draw a well-conditioned P")
    A1 = P @ B @ np.linalg.inv(P)
    U = P.astype(np.complex128) @ _block_pair_eigvecs(npairs)
    V = np.linalg.inv(U)
    lam = np.empty(n, dtype=np.complex128)
    lam[0::2] = s + 1j * w
    lam[1::2] = s - 1j * w
    resid = np.abs(V @ U - np.eye(n)).max()
    if resid > 1e-12:  # pragma: no cover
        raise RuntimeError(f"V U - I too large: {resid}")
    return ModalSystem(n=n, A1=A1, lam=lam, U=U, V=V, P=P)


def random_packed_tensor(n: int, N: int, seed: int, density: float = 0.30) -> np.ndarray:
    """Packed symmetric A_N: a fraction `density` of the unique entries is N(0,1), the rest 0."""
    rng = np.random.default_rng(seed)
    m = packed_count(n, N)
    vals = rng.standard_normal((n, m))
    keep = rng.random((n, m)) < density
    return np.ascontiguousarray(np.where(keep, vals, 0.0))


def random_packed_tensor_dense_fill(n: int, N: int, seed: int) -> np.ndarray:
    """Packed symmetric A_N with every unique entry N(0,1)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, packed_count(n, N))))


# ----------------------------------------------------------------------------------------
# Named workloads.
# ----------------------------------------------------------------------------------------

def config_small(seed: int = 0, orders=(2, 3)) -> ModalSystem:
    """n = 10 (5 conjugate mode pairs), dense P, A2/A3 30% nonzero N(0,1)."""
    sysm = modal_system(10, seed, block=2)
    for N in orders:
        sysm.tensors[N] = random_packed_tensor(10, N, seed * 1000 + N)
    return sysm


def config_blocks(n: int, seed: int = 0, orders=(2, 3, 4)) -> ModalSystem:
    """n states as n/4 generator-like blocks of 4 states with 10% sparse inter-block coupling
    N(0, 0.1); A_N 30% nonzero N(0,1)."""
    sysm = modal_system(n, seed, block=4, coupling=0.1, coupling_density=0.10)
    for N in orders:
        sysm.tensors[N] = random_packed_tensor(n, N, seed * 1000 + N)
    return sysm


def config_n60(seed: int = 0, orders=(2, 3, 4)) -> ModalSystem:
    return config_blocks(60, seed, orders)


def config_n120(seed: int = 0, orders=(3, 4)) -> ModalSystem:
    return config_blocks(120, seed, orders)


def near_resonant_system(n: int, seed: int, frac_rungs: float = 0.22,
                         detune: float = 3e-4) -> ModalSystem:
    """Eigenvalues with a harmonic ladder lambda_m = m*lambda0 + delta_m (|delta_m| <= detune) on a
    fraction of the conjugate pairs, so that lambda_a + lambda_b - lambda_{a+b} is within ~1e-3 of
    zero for every rung pair with a + b on the ladder; remaining pairs as in modal_system."""
    rng = np.random.default_rng(seed + 7919)
    npairs = n // 2
    L = max(2, int(round(frac_rungs * n)))
    L = min(L, npairs)
    s0 = rng.uniform(-2.0 / L, -0.05)
    s0 = min(s0, -0.05 / 1.0)
    w0 = rng.uniform(0.5, 15.0 / L)
    s = rng.uniform(*SIGMA_RANGE, size=npairs)
    w = rng.uniform(*OMEGA_RANGE, size=npairs)
    m = np.arange(1, L + 1)
    s[:L] = m * s0 + rng.uniform(-detune, detune, size=L)
    w[:L] = m * w0 + rng.uniform(-detune, detune, size=L)
    s[:L] = np.clip(s[:L], -50.0, -1e-3)
    return modal_system(n, seed, block=2, sigmas=s, omegas=w)


def resonance_fraction(lam: np.ndarray, tol: float = 1e-3) -> float:
    """Fraction of ordered (r, s) pairs that have some i with |lam_r + lam_s - lam_i| < tol."""
    S = lam[:, None] + lam[None, :]
    d = np.abs(S[:, :, None] - lam[None, None, :]).min(axis=2)
    return float((d < tol).mean())


def batch_systems(count: int = 256, seed: int = 0, n_lo: int = 20, n_hi: int = 80,
                  orders=(2, 3)):
    """`count` systems of uneven size n ~ U{n_lo..n_hi} (even) and order drawn from `orders`."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_lo // 2, n_hi // 2 + 1)) * 2
        N = int(rng.choice(orders))
        sysm = near_resonant_system(n, seed * 100003 + b)
        sysm.tensors[N] = random_packed_tensor(n, N, seed * 100003 + b * 7 + N)
        out.append((sysm, N))
    return out


# ----------------------------------------------------------------------------------------
# Parameterised family of operating points (learned-surrogate workload).
# ----------------------------------------------------------------------------------------

@dataclass
class OperatingPointFamily:
    """A1(p) = A0 + (s - 1) A_load + sum_c (g_c - 1) A_ctrl[c] for p = (s, g_1, g_2, g_3); the
    Taylor tensors do not depend on p."""
    n: int
    A0: np.ndarray           # real [n, n]
    A_load: np.ndarray       # real [n, n]
    A_ctrl: np.ndarray       # real [3, n, n]
    tensors: dict            # order -> packed float64
    lo: np.ndarray           # [4] parameter lower bounds
    hi: np.ndarray           # [4] parameter upper bounds
    p0: np.ndarray           # [4] nominal operating point

    def A(self, p) -> np.ndarray:
        p = np.asarray(p, dtype=np.float64)
        return (self.A0 + (p[0] - 1.0) * self.A_load
                + np.tensordot(p[1:] - 1.0, self.A_ctrl, axes=1))


def surrogate_family(n: int = 40, seed: int = 0, orders=(2, 3),
                     load_scale: float = 0.05, ctrl_scale: float = 0.05) -> OperatingPointFamily:
    """n states in n/4 generator-like blocks (as config_blocks). The load matrix perturbs every
    4x4 diagonal block with N(0, load_scale) entries; controller c perturbs the diagonal blocks
    b with b % 3 == c with N(0, ctrl_scale) entries. Load scale s ~ U[0.6, 1.2], gains
    g_c ~ U[0.5, 2]; nominal point (1, 1, 1, 1). Tensors A_N 30% nonzero N(0, 1)."""
    base = modal_system(n, seed, block=4, coupling=0.1, coupling_density=0.10)
    rng = np.random.default_rng(seed + 104729)
    nb = n // 4
    A_load = np.zeros((n, n))
    A_ctrl = np.zeros((3, n, n))
    for b in range(nb):
        sl = slice(4 * b, 4 * b + 4)
        A_load[sl, sl] = load_scale * rng.standard_normal((4, 4))
        A_ctrl[b % 3][sl, sl] = ctrl_scale * rng.standard_normal((4, 4))
    tensors = {N: random_packed_tensor(n, N, seed * 1000 + 500 + N) for N in orders}
    return OperatingPointFamily(n=n, A0=base.A1, A_load=A_load, A_ctrl=A_ctrl, tensors=tensors,
                                lo=np.array([0.6, 0.5, 0.5, 0.5]),
                                hi=np.array([1.2, 2.0, 2.0, 2.0]),
                                p0=np.ones(4))


def operating_points(fam: OperatingPointFamily, count: int, seed: int) -> np.ndarray:
    """`count` parameter vectors drawn uniformly from the family's box, [count, 4]."""
    rng = np.random.default_rng(seed)
    return fam.lo + (fam.hi - fam.lo) * rng.random((count, 4))


# ----------------------------------------------------------------------------------------
# Multi-machine swing model (power-system-shaped inputs with closed-form derivatives).
# ----------------------------------------------------------------------------------------

@dataclass
class SwingModel:
    """m machines, states x = (delta_0..delta_{m-1}, omega_0..omega_{m-1}):
    d delta_j/dt = omega_j,
    d omega_j/dt = (P_j - D_j omega_j - sum_k V_j V_k (G_jk cos(d_j - d_k) + B_jk sin(d_j - d_k)))
                   / (2 H_j),
    with P_j chosen so that the angles `delta` (and omega = 0) are an equilibrium."""
    m: int
    H: np.ndarray
    D: np.ndarray
    V: np.ndarray
    delta: np.ndarray
    G: np.ndarray      # [m, m], symmetric, zero diagonal
    B: np.ndarray      # [m, m], symmetric, zero diagonal
    P: np.ndarray
    Gb: np.ndarray     # [m] lines to a reference bus (voltage 1, angle 0)
    Bb: np.ndarray

    def f(self, x):
        x = np.asarray(x, dtype=np.float64)
        m = self.m
        d, w = x[:m], x[m:]
        t = d[:, None] - d[None, :]
        net = (self.V[:, None] * self.V[None, :] * (self.G * np.cos(t) + self.B * np.sin(t))).sum(1)
        net = net + self.V * (self.Gb * np.cos(d) + self.Bb * np.sin(d))
        return np.concatenate([w, (self.P - self.D * w - net) / (2.0 * self.H)])

    def jacobian(self):
        """A1 at the equilibrium (closed form)."""
        m = self.m
        t = self.delta[:, None] - self.delta[None, :]
        gp = self.V[:, None] * self.V[None, :] * (-self.G * np.sin(t) + self.B * np.cos(t))
        np.fill_diagonal(gp, 0.0)
        bus = self.V * (-self.Gb * np.sin(self.delta) + self.Bb * np.cos(self.delta))
        A = np.zeros((2 * m, 2 * m))
        A[:m, m:] = np.eye(m)
        A[m:, :m] = (gp - np.diag(gp.sum(1) + bus)) / (2.0 * self.H)[:, None]
        A[m:, m:] = -np.diag(self.D / (2.0 * self.H))
        return A


def swing_model(m: int, seed: int = 0, bus: bool = True) -> SwingModel:
    """A ring of m machines plus random extra lines (about two per machine); line susceptances
    U[5, 15], conductances U[0, 1]; inertia H ~ U[2, 8], damping D ~ U[0.5, 2], voltages
    U[0.95, 1.05], angles N(0, 0.2); with `bus`, every third machine also has a line to a
    reference bus (susceptance U[5, 15], conductance U[0, 1]), which removes the rotational zero
    mode (without it the modes include lambda = 0 and the denominators lambda_0 + lambda_p -
    lambda_p vanish exactly)."""
    rng = np.random.default_rng(seed + 911)
    B = np.zeros((m, m))
    G = np.zeros((m, m))
    edges = {(j, (j + 1) % m) for j in range(m)} if m > 2 else {(0, 1)}
    for _ in range(2 * m):
        a, b = rng.integers(0, m, 2)
        if a != b:
            edges.add((min(a, b), max(a, b)))
    for a, b in edges:
        a, b = min(a, b), max(a, b)
        B[a, b] = B[b, a] = rng.uniform(5.0, 15.0)
        G[a, b] = G[b, a] = rng.uniform(0.0, 1.0)
    H = rng.uniform(2.0, 8.0, m)
    D = rng.uniform(0.5, 2.0, m)
    V = rng.uniform(0.95, 1.05, m)
    delta = rng.normal(0.0, 0.2, m)
    Gb = np.zeros(m)
    Bb = np.zeros(m)
    if bus:
        for j in range(0, m, 3):
            Bb[j] = rng.uniform(5.0, 15.0)
            Gb[j] = rng.uniform(0.0, 1.0)
    t = delta[:, None] - delta[None, :]
    P = (V[:, None] * V[None, :] * (G * np.cos(t) + B * np.sin(t))).sum(1)
    P = P + V * (Gb * np.cos(delta) + Bb * np.sin(delta))
    return SwingModel(m=m, H=H, D=D, V=V, delta=delta, G=G, B=B, P=P, Gb=Gb, Bb=Bb)


def swing_system(model: SwingModel) -> ModalSystem:
    """Eigen-triple of the swing model's linearisation (LAPACK through NumPy), V = U^-1."""
    A1 = model.jacobian()
    lam, U = np.linalg.eig(A1)
    V = np.linalg.inv(U)
    return ModalSystem(n=2 * model.m, A1=A1, lam=lam.astype(np.complex128),
                       U=U.astype(np.complex128), V=V.astype(np.complex128), P=np.eye(2 * model.m))
