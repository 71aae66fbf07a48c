"""GB300 library for high-order nonlinear participation factors (arXiv 2509.08968).

Thin ctypes binding over the C ABI in include/npf.h (libnpf.so, built in-tree by
``paper_2509_08968_gb300.build``). Every step of the computation runs in the library's CUDA
kernels; this module only marshals arguments. Arrays may be NumPy arrays (host) or CUDA torch
tensors (device pointers are passed straight through). There is no CPU fallback: if the shared
library is missing the import of the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpf.so")

# status codes / options / precisions (mirrors include/npf.h)
NPF_OK = 0
NPF_ERR_ARG = 1
NPF_ERR_NOT_INVERSE = 2
NPF_ERR_OOM = 3
NPF_ERR_MISSING_TENSOR = 4
NPF_ERR_CUDA = 5
NPF_ERR_TIMEOUT = 6
NPF_ERR_UNSUPPORTED = 7

(OPT_PRECISION, OPT_EPS, OPT_STREAM, OPT_SLICES, OPT_DIVIDE, OPT_MEM_BUDGET, OPT_PROFILE,
 OPT_TILE_N, OPT_FP64_QUOTIENT, OPT_DEBUG_STALL) = range(10)
PREC_FP64, PREC_SPLIT_BF16, PREC_FP32 = 0, 1, 2
PRECISIONS = {"fp64": PREC_FP64, "split_bf16": PREC_SPLIT_BF16, "fp32": PREC_FP32}

_lib = None


class NpfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"npf status {status}: {msg}")
        self.status = status


def load():
    """Load libnpf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2509_08968_gb300.build` "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd, i64, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                           ctypes.c_size_t)
    lib.npf_plan.restype = vp
    lib.npf_plan.argtypes = [ci, ci, vp, vp, vp, sz]
    lib.npf_set_tensor.argtypes = [vp, ci, vp]
    lib.npf_set_modes.argtypes = [vp, vp, vp, vp]
    lib.npf_set_mode_subset.argtypes = [vp, ci, vp]
    lib.npf_mlp_create.restype = vp
    lib.npf_mlp_create.argtypes = [ci, ci, vp, vp, vp]
    lib.npf_mlp_param_count.restype = i64
    lib.npf_mlp_param_count.argtypes = [vp]
    lib.npf_mlp_get_weights.argtypes = [vp, vp]
    lib.npf_mlp_forward.argtypes = [vp, ci, vp, vp]
    lib.npf_mlp_loss_grad.argtypes = [vp, ci, vp, vp, vp, vp]
    lib.npf_mlp_train.argtypes = [vp, ci, vp, vp, ci, ci, cd, ctypes.c_uint64, vp]
    lib.npf_mlp_predict.argtypes = [vp, ci, vp, vp, vp, cd, vp, vp, vp]
    lib.npf_mlp_destroy.argtypes = [vp]
    lib.npf_mlp_destroy.restype = None
    lib.npf_compute.argtypes = [vp, ci, vp]
    lib.npf_compute_prefetch.argtypes = [vp, ci, vp, ci, vp, vp]
    lib.npf_destroy.argtypes = [vp]
    lib.npf_destroy.restype = None
    lib.npf_set_option.argtypes = [vp, ci, cd]
    lib.npf_get_term.argtypes = [vp, ci, vp]
    lib.npf_get_modal_slab.argtypes = [vp, ci, vp, vp]
    lib.npf_interaction.argtypes = [vp, ci, cd, vp]
    lib.npf_get_term_rows.argtypes = [vp, ci, ci, ci, vp]
    lib.npf_finish_terms.argtypes = [vp, ci, vp, vp]
    lib.npf_set_tensor_swing.argtypes = [vp, ci, vp, vp, vp, vp, vp, vp, vp]
    lib.npf_get_tensor.argtypes = [vp, ci, vp]
    lib.npf_batch_compute.argtypes = [ci, vp, vp, vp]
    lib.npf_last_error.restype = ctypes.c_char_p
    lib.npf_last_status.restype = ci
    lib.npf_alg1_batches.restype = i64
    lib.npf_alg1_batches.argtypes = [ci, ci, cd, ci, vp, vp, vp, vp]
    lib.npf_get_profile.argtypes = [vp, ci, vp, vp, vp, ci]
    lib.npf_launch_count.restype = i64
    lib.npf_launch_count.argtypes = []
    lib.npf_tuned_tile.restype = ci
    lib.npf_tuned_tile.argtypes = [ci, ci, ci, ci, ci]
    _lib = lib
    return lib


def _check(rc):
    if rc != NPF_OK:
        raise NpfError(rc, load().npf_last_error().decode(errors="replace"))


def _ptr(a):
    """Pointer of a NumPy array or a torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _host_c128(a):
    a = np.asarray(a, dtype=np.complex128)
    return np.ascontiguousarray(a)


def _is_torch(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


class Plan:
    """One system: eigenvalues `lam` [n], right eigenvectors U [n, n] (columns), left
    eigenvectors V = U^-1 [n, n] (rows), Taylor orders up to N_max."""

    def __init__(self, lam, U, V, N_max, mem_budget=0, precision="split_bf16", stream=None):
        lib = load()
        self._keep = []
        self._prefetched = []   # arrays whose prefetch copies the next tensor-using call waits for
        if _is_torch(lam):
            n = int(lam.shape[0])
            args = (lam, U, V)
        else:
            lam, U, V = _host_c128(lam), _host_c128(U), _host_c128(V)
            n = lam.shape[0]
            args = (lam, U, V)
        self.n = n
        self.N_max = N_max
        h = lib.npf_plan(n, N_max, _ptr(args[0]), _ptr(args[1]), _ptr(args[2]), int(mem_budget))
        if not h:
            raise NpfError(lib.npf_last_status(), lib.npf_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)
        self.set_precision(precision)
        if stream is not None:
            self.set_option(OPT_STREAM, float(stream))

    # -- options ---------------------------------------------------------------------------
    def set_option(self, key, value):
        _check(load().npf_set_option(self._h, key, float(value)))

    def set_precision(self, precision):
        self.set_option(OPT_PRECISION, PRECISIONS[precision] if isinstance(precision, str)
                        else precision)

    def set_stream(self, stream):
        """cudaStream_t as an integer (torch: stream.cuda_stream)."""
        self.set_option(OPT_STREAM, float(stream))

    # -- data ------------------------------------------------------------------------------
    def set_modes(self, lam, U, V):
        """Replace the modal data by another system of the same size (buffers kept)."""
        if not _is_torch(lam):
            lam, U, V = _host_c128(lam), _host_c128(U), _host_c128(V)
        _check(load().npf_set_modes(self._h, _ptr(lam), _ptr(U), _ptr(V)))

    def set_mode_subset(self, modes=None):
        """Restrict the modal indices to `modes` (None or all modes: no restriction)."""
        if modes is None:
            _check(load().npf_set_mode_subset(self._h, 0, None))
            return
        m = np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
        _check(load().npf_set_mode_subset(self._h, int(m.size), _ptr(m)))

    def set_tensor(self, order, coeffs):
        """Packed symmetric order-`order` tensor [n, C(n+order-1, order)] float64."""
        if not _is_torch(coeffs):
            coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
        _check(load().npf_set_tensor(self._h, order, _ptr(coeffs)))
        self._prefetched = []

    def set_tensor_swing(self, order, model):
        """Generate the order-`order` tensor of a swing model on the GPU (model: H, V, delta,
        G, B, Gb, Bb as float64 arrays; n = 2 * len(H))."""
        arrs = [np.ascontiguousarray(np.asarray(getattr(model, k), dtype=np.float64))
                for k in ("H", "V", "delta", "G", "B", "Gb", "Bb")]
        _check(load().npf_set_tensor_swing(self._h, order, *[_ptr(a) for a in arrs]))
        self._prefetched = []

    def get_tensor(self, order):
        """The plan's packed order-`order` tensor [n, C(n+order-1, order)]."""
        from math import comb
        out = np.empty((self.n, comb(self.n + order - 1, order)), dtype=np.float64)
        _check(load().npf_get_tensor(self._h, order, _ptr(out)))
        self._prefetched = []
        return out

    def compute(self, order, out=None):
        """NPF of the given order; returns a NumPy complex128 [n, n] (or fills `out`, which may
        be a complex128 CUDA tensor or NumPy array)."""
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        _check(load().npf_compute(self._h, order, _ptr(out)))
        self._prefetched = []
        return out

    def compute_prefetch(self, order, out=None, next_tensors=None):
        """compute(order, out) while the packed tensors of `next_tensors` ({order: tensor}, host
        or device) upload on the plan's upload stream; they replace the current tensors of those
        orders at the next call that uses tensors, and stay referenced until that call returns."""
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        items = []
        for N, t in (next_tensors or {}).items():
            if not _is_torch(t):
                t = np.ascontiguousarray(t, dtype=np.float64)
            items.append((int(N), t))
        orders = (ctypes.c_int * max(1, len(items)))(*[N for N, _ in items])
        ptrs = (ctypes.c_void_p * max(1, len(items)))(*[_ptr(t).value for _, t in items])
        pending = self._prefetched
        self._prefetched = pending + [t for _, t in items]   # until the call has returned
        _check(load().npf_compute_prefetch(self._h, order, _ptr(out), len(items), orders, ptrs))
        self._prefetched = [t for _, t in items]   # the previous ones were waited for
        return out

    def term(self, order, out=None):
        """Order-only correction Psi_N[i, k]."""
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        _check(load().npf_get_term(self._h, order, _ptr(out)))
        self._prefetched = []
        return out

    def interaction(self, order, delta, out=None):
        """Mode-interaction NPFs [order, n, n]: [0] = pN1, [M-1] = pNM (Eqs. 6-9) for the
        excitation delta e_k of each state k."""
        if out is None:
            out = np.empty((order, self.n, self.n), dtype=np.complex128)
        _check(load().npf_interaction(self._h, order, float(delta), _ptr(out)))
        self._prefetched = []
        return out

    def term_rows(self, order, i_lo, i_hi, out=None):
        """Rows [i_lo, i_hi) of Psi_N (other rows zero)."""
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        _check(load().npf_get_term_rows(self._h, order, int(i_lo), int(i_hi), _ptr(out)))
        self._prefetched = []
        return out

    def finish_terms(self, terms, out=None):
        """NPF from given correction terms (Alg. 2 step 20): `terms` is one Psi_N array [n, n]
        or a stack [count, n, n] (NumPy or CUDA torch, complex128)."""
        if not _is_torch(terms):
            terms = np.ascontiguousarray(np.asarray(terms, dtype=np.complex128))
        count = 1 if len(terms.shape) == 2 else int(terms.shape[0])
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        _check(load().npf_finish_terms(self._h, count, _ptr(terms), _ptr(out)))
        self._prefetched = []
        return out

    def modal_slab(self, order, prefix, out=None):
        """h^i_{prefix, q} as [n (i), n (q)]."""
        pre = np.ascontiguousarray(np.asarray(prefix, dtype=np.int32))
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.complex128)
        _check(load().npf_get_modal_slab(self._h, order, _ptr(pre), _ptr(out)))
        self._prefetched = []
        return out

    def profile(self, reset=False):
        """{kernel name: (launches, total ms)} recorded while OPT_PROFILE is 1."""
        lib = load()
        cap = 64
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        k = lib.npf_get_profile(self._h, cap, names, launches, ms, 1 if reset else 0)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(k, cap))}

    def close(self):
        if getattr(self, "_h", None):
            load().npf_destroy(self._h)   # waits for the plan's streams
            self._h = None
        self._prefetched = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_compute(plans, orders, outs):
    """NPF_{orders[b]} of plans[b] into outs[b] (NumPy or CUDA tensors) in one call."""
    lib = load()
    count = len(plans)
    hp = (ctypes.c_void_p * count)(*[p._h.value for p in plans])
    od = (ctypes.c_int * count)(*orders)
    op = (ctypes.c_void_p * count)(*[_ptr(o).value for o in outs])
    _check(lib.npf_batch_compute(count, hp, od, op))
    for p in plans:
        p._prefetched = []
    return outs


def alg1_batches(n_dim, n_s, m_limit_gb, bytes_per_elem=8):
    """Algorithm 1 sizing: returns dict(BC, max_batch, batches, total_gb, per_batch_gb)."""
    lib = load()
    BC = (ctypes.c_int64 * n_dim)()
    MB = (ctypes.c_int64 * n_dim)()
    tot = ctypes.c_double()
    per = ctypes.c_double()
    nb = lib.npf_alg1_batches(n_dim, n_s, float(m_limit_gb), bytes_per_elem, BC, MB,
                              ctypes.byref(tot), ctypes.byref(per))
    if nb < 0:
        raise NpfError(NPF_ERR_ARG, "bad Algorithm 1 arguments")
    return dict(BC=list(BC), max_batch=list(MB), batches=int(nb), total_gb=tot.value,
                per_batch_gb=per.value)


def launch_count():
    return int(load().npf_launch_count())


def tuned_tile(n, order, precision="split_bf16", slices=0, divide=True):
    """Tile width the autotuner chose for this key in this process (0 = not tuned yet)."""
    pr = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return int(load().npf_tuned_tile(n, order, pr, slices, 1 if divide else 0))
