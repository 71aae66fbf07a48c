"""CPU oracle for the NPF computation (test infrastructure only).

Loads the plain-C complex128 implementation in npf_oracle.c (compiled here with gcc into
oracle/_build/) through ctypes. Only tests/, the package smoke check and the benchmark's
CPU-baseline leg may import this package; the library never does.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libnpf_oracle.so")
_lock = threading.Lock()
_lib = None


_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fcx-limited-range",
           "-fno-fast-math"]


def compile_source(src: str, out: str) -> str:
    """Compile a C source of the oracle's interface with the oracle's own flags into `out`."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *_CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile npf_oracle.c with gcc (-O2, OpenMP, no fast-math) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_source(_SRC, _SO)
    return _SO


def _bind(lib):
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    cdbl = ctypes.c_double
    vp = ctypes.c_void_p
    lib.npfo_packed_count.restype = i64
    lib.npfo_packed_count.argtypes = [ci, ci]
    lib.npfo_unpack.argtypes = [ci, ci, vp, vp]
    lib.npfo_h_brute.argtypes = [ci, ci, vp, vp, vp, vp, cdbl, ci, vp]
    lib.npfo_psiN_brute.argtypes = [ci, ci, vp, vp, vp]
    lib.npfo_h_fact.argtypes = [ci, ci, vp, vp, vp, vp, cdbl, ci, ci, ci, vp]
    lib.npfo_psiN_accumulate.argtypes = [ci, ci, vp, vp, ci, ci, vp]
    lib.npfo_psiN.argtypes = [ci, ci, vp, vp, vp, vp, cdbl, ci, ci, vp]
    lib.npfo_h_slab.argtypes = [ci, ci, vp, vp, vp, vp, cdbl, ci, vp, vp]
    lib.npfo_npf.argtypes = [ci, vp, vp, vp, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


@contextlib.contextmanager
def substituted_library(so_path: str):
    """Run the oracle's functions on another compiled copy of its C source (a test that plants
    a mistake in the oracle checks that the pins catch it); the own library is restored after."""
    global _lib
    own = _load()
    with _lock:
        _lib = _bind(ctypes.CDLL(os.path.abspath(so_path)))
    try:
        yield
    finally:
        with _lock:
            _lib = own


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


DEFAULT_EPS = 1e-8


def packed_count(n: int, N: int) -> int:
    return int(_load().npfo_packed_count(n, N))


def unpack(packed, n: int, N: int) -> np.ndarray:
    """Dense [n, n, .., n] (upper index first) from the packed symmetric tensor."""
    packed = _f64(packed)
    out = np.empty((n,) + (n,) * N, dtype=np.float64)
    _load().npfo_unpack(n, N, _p(packed), _p(out))
    return out


def h_brute(dense, U, V, lam, eps=DEFAULT_EPS, divide=True) -> np.ndarray:
    """Eq. 4 literally over every index. dense has shape (n,)*(N+1). Returns h [n]*(N+1)."""
    dense = _f64(dense)
    n = dense.shape[0]
    N = dense.ndim - 1
    U, V, lam = _c128(U), _c128(V), _c128(lam)
    h = np.empty((n,) * (N + 1), dtype=np.complex128)
    _load().npfo_h_brute(n, N, _p(dense), _p(U), _p(V), _p(lam), eps, 0 if divide else 1, _p(h))
    return h


def psiN_brute(h, V) -> np.ndarray:
    h = _c128(h)
    n = h.shape[0]
    N = h.ndim - 1
    V = _c128(V)
    out = np.empty((n, n), dtype=np.complex128)
    _load().npfo_psiN_brute(n, N, _p(h), _p(V), _p(out))
    return out


def h_fact(packed, n, N, U, V, lam, eps=DEFAULT_EPS, divide=True, p1_lo=0, p1_hi=None):
    """h^i_{p_1..p_N} for p_1 in [p1_lo, p1_hi) by the factorised contraction order of Alg. 2.
    Returns an array [n, p1_hi-p1_lo, n, .., n]."""
    if p1_hi is None:
        p1_hi = n
    packed = _f64(packed)
    U, V, lam = _c128(U), _c128(V), _c128(lam)
    out = np.empty((n, p1_hi - p1_lo) + (n,) * (N - 1), dtype=np.complex128)
    _load().npfo_h_fact(n, N, _p(packed), _p(U), _p(V), _p(lam), eps, 0 if divide else 1,
                        p1_lo, p1_hi, _p(out))
    return out


def psiN(packed, n, N, U, V, lam, eps=DEFAULT_EPS, divide=True, p1_block=1) -> np.ndarray:
    """Psi_N[i, k] (the order-N correction term of Eq. 7 for x(0) = e_k)."""
    packed = _f64(packed)
    U, V, lam = _c128(U), _c128(V), _c128(lam)
    out = np.empty((n, n), dtype=np.complex128)
    _load().npfo_psiN(n, N, _p(packed), _p(U), _p(V), _p(lam), eps, 0 if divide else 1,
                      p1_block, _p(out))
    return out


def psiN_partial(packed, n, N, U, V, lam, p1_lo, p1_hi, eps=DEFAULT_EPS, divide=True):
    """The share of Psi_N contributed by output indices p_1 in [p1_lo, p1_hi)."""
    hb = h_fact(packed, n, N, U, V, lam, eps, divide, p1_lo, p1_hi)
    acc = np.zeros((n, n), dtype=np.complex128)
    _load().npfo_psiN_accumulate(n, N, _p(hb), _p(_c128(V)), p1_lo, p1_hi, _p(acc))
    return acc


def h_slab(packed, n, N, U, V, lam, prefix, eps=DEFAULT_EPS, divide=True) -> np.ndarray:
    """h^i_{prefix, q} for every i and q: array [n (i), n (q)]."""
    packed = _f64(packed)
    U, V, lam = _c128(U), _c128(V), _c128(lam)
    pre = np.ascontiguousarray(np.asarray(prefix, dtype=np.int32))
    assert pre.size == N - 1
    out = np.empty((n, n), dtype=np.complex128)
    _load().npfo_h_slab(n, N, _p(packed), _p(U), _p(V), _p(lam), eps, 0 if divide else 1,
                        _p(pre), _p(out))
    return out


def npf(U, V, S=None) -> np.ndarray:
    """NPF[k, i] = phi_{k i} (psi_{i k} + S[i, k]); S = sum of Psi_N terms (None: linear PFs)."""
    U, V = _c128(U), _c128(V)
    n = U.shape[0]
    out = np.empty((n, n), dtype=np.complex128)
    Sp = None if S is None else _c128(S)
    _load().npfo_npf(n, _p(U), _p(V), None if Sp is None else _p(Sp), _p(out))
    return out


def npf_orders(sysm, order, eps=DEFAULT_EPS, p1_block=1):
    """NPF of the given order: linear PFs plus Psi_m of every order 2..order present in
    sysm.tensors (Alg. 2 step 20, cumulative)."""
    n = sysm.n
    S = np.zeros((n, n), dtype=np.complex128)
    for m in range(2, order + 1):
        if m in sysm.tensors:
            S += psiN(sysm.tensors[m], n, m, sysm.U, sysm.V, sysm.lam, eps, True, p1_block)
    return npf(sysm.U, sysm.V, S)


def reduce_weights(packed, n, N, U, V, lam, W, eps=DEFAULT_EPS, divide=True, p1_block=None):
    """T[i, k] = sum_p h^i_p prod_m W[p_m, k]: the contraction of steps 12-19 with weight columns
    W[:, k] in place of Psi[:, k] (h from the factorised form, with Psi on the upper index)."""
    W = _c128(W)
    p1_block = n if p1_block is None else p1_block
    acc = np.zeros((n, n), dtype=np.complex128)
    for lo in range(0, n, p1_block):
        hi = min(n, lo + p1_block)
        hb = h_fact(packed, n, N, U, V, lam, eps, divide, lo, hi)
        _load().npfo_psiN_accumulate(n, N, _p(hb), _p(W), lo, hi, _p(acc))
    return -acc


def interaction_npfs(sysm, order, delta, eps=DEFAULT_EPS, p1_block=None):
    """Mode-interaction NPFs of the excitation x(0) = delta e_k (Eqs. 6-9), [order, n, n]:
    [0][k, i] = pN1 = phi_ki z^i(0) with z(0) = zeta - sum_N hN(zeta..zeta), zeta = delta Psi[:, k]
    (Eq. 7; Psi_N as computed by psiN already carries the minus sign); [M-1][k, i] = pNM =
    phi_ki sum_p hM^i_p prod_m zeta*_{p_m} with zeta* = z(0) (Eqs. 8-9), zero without an order-M
    tensor."""
    n = sysm.n
    U, V = _c128(sysm.U), _c128(sysm.V)
    z = delta * V
    for N in range(2, order + 1):
        if N in sysm.tensors:
            z = z + delta ** N * psiN(sysm.tensors[N], n, N, U, V, sysm.lam, eps, True,
                                      p1_block or n)
    out = np.zeros((order, n, n), dtype=np.complex128)
    out[0] = U * z.T
    for M in range(2, order + 1):
        if M in sysm.tensors:
            T = reduce_weights(sysm.tensors[M], n, M, U, V, sysm.lam, z, eps, True, p1_block)
            out[M - 1] = U * T.T
    return out


def psiN_subset(packed, n, N, U, V, lam, modes, eps=DEFAULT_EPS, p1_block=None):
    """Psi_N restricted to a set of modes: for i in `modes`,
    -sum_{p in modes^N} h^i_p prod_m psi_{p_m k} (the sums of Eq. 7 over the subset only); rows of
    the other modes are zero. h^i_p itself does not depend on the subset (Eq. 4)."""
    modes = np.asarray(modes)
    W = np.zeros((n, n), dtype=np.complex128)
    W[modes] = _c128(V)[modes]
    T = reduce_weights(packed, n, N, U, V, lam, W, eps, True, p1_block)
    out = np.zeros((n, n), dtype=np.complex128)
    out[modes] = -T[modes]
    return out
