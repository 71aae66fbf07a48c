"""The allocation-free entry point npf_term_fp64_noalloc, called through the C ABI.

Some callers may not allocate device memory: a process confined to a memory pool it was handed, a
plugin whose host application forbids cudaMalloc, a latency-bound loop that cannot take the
device-wide synchronisation an allocation may imply. For them the library offers one entry point
whose scratch is a fixed 64 MiB device array. This test checks its output against the CPU oracle
and against the allocating entry point (npf_plan + npf_get_term, native FP64) on consecutive calls
with different sizes, so that each call runs on the array as the previous one left it; one case
(n = 30, order 4) needs two output-index batches per pass through the array. It also checks that a
problem too large for the array is rejected.
"""
import ctypes

import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-12          # the native-FP64 parity tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def lib():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as npf
    L = npf.load()
    vp = ctypes.c_void_p
    L.npf_term_fp64_noalloc.restype = ctypes.c_int
    L.npf_term_fp64_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                        ctypes.c_double, vp, vp]
    return npf, L


def _noalloc_term(npf, L, sysm, N, eps=1e-8):
    import torch
    dev = torch.device("cuda", 0)
    lam = torch.from_numpy(np.ascontiguousarray(sysm.lam)).to(dev)
    U = torch.from_numpy(np.ascontiguousarray(sysm.U)).to(dev)
    V = torch.from_numpy(np.ascontiguousarray(sysm.V)).to(dev)
    A = torch.from_numpy(np.ascontiguousarray(sysm.tensors[N])).to(dev)
    out = torch.full((sysm.n, sysm.n), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    rc = L.npf_term_fp64_noalloc(sysm.n, N, lam.data_ptr(), U.data_ptr(), V.data_ptr(),
                                 A.data_ptr(), eps, out.data_ptr(), None)
    assert rc == npf.NPF_OK, L.npf_last_error().decode()
    return out.cpu().numpy()


def _reference_term(npf, sysm, N):
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N, precision="fp64") as p:
        p.set_tensor(N, sysm.tensors[N])
        return p.term(N)


def _system_n30():
    sysm = S.modal_system(30, 7)
    sysm.tensors[4] = S.random_packed_tensor(30, 4, 7)
    return sysm


def test_noalloc_matches_oracle_and_allocating_entry_point(lib):
    npf, L = lib
    cases = ((S.config_blocks(20, 5, orders=(3,)), 3),
             (_system_n30(), 4),                      # 2 batches of p_1 per pass (26 MB each)
             (S.config_small(1, orders=(2, 3)), 3))
    for sysm, N in cases:
        got = _noalloc_term(npf, L, sysm, N)
        assert np.isfinite(got).all()
        ref = oracle.psiN(sysm.tensors[N], sysm.n, N, sysm.U, sysm.V, sysm.lam)
        assert rel_fro(got, ref) < TOL, (sysm.n, N)
        assert rel_fro(got, _reference_term(npf, sysm, N)) < TOL, (sysm.n, N)


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    npf, L = lib
    import torch
    n, N = 60, 4                     # 2 n^4 complex = 415 MB of scratch > 64 MiB
    dummy = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    rc = L.npf_term_fp64_noalloc(n, N, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 dummy.data_ptr(), 1e-8, dummy.data_ptr(), None)
    assert rc == npf.NPF_ERR_UNSUPPORTED
    assert b"64 MiB" in L.npf_last_error()
