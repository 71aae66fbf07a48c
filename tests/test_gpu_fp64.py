"""Native-FP64 GPU form against the CPU oracle (and error behaviour of the ABI)."""
import itertools
import math

import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import make_plan, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_system_orders_2_3(npf, seed):
    sysm = S.config_small(seed, orders=(2, 3))
    with make_plan(npf, sysm, 3, "fp64") as p:
        for N in (2, 3):
            ref = oracle.psiN(sysm.tensors[N], 10, N, sysm.U, sysm.V, sysm.lam, p1_block=10)
            assert rel_fro(p.term(N), ref) < TOL
        np.testing.assert_allclose(p.compute(1), sysm.U * sysm.V.T, rtol=1e-14, atol=1e-15)
        ref = oracle.npf_orders(sysm, 3, p1_block=10)
        assert rel_fro(p.compute(3), ref) < TOL


@pytest.mark.parametrize("n,N", [(6, 4), (4, 5), (2, 6)])
def test_high_orders_small_n(npf, n, N):
    sysm = S.modal_system(n, 3 * n + N)
    sysm.tensors[N] = S.random_packed_tensor(n, N, 17 + N)
    with make_plan(npf, sysm, N, "fp64") as p:
        ref = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=n)
        assert rel_fro(p.term(N), ref) < TOL


def test_batched_output_index_matches_single_batch(npf):
    sysm = S.config_blocks(20, 5, orders=(3,))
    with make_plan(npf, sysm, 3, "fp64") as p:
        one = p.term(3)
        p.set_option(npf.OPT_MEM_BUDGET, (2 * 20 ** 3 + 20 ** 2) * 16 * 3)   # batches of 3 values
        many = p.term(3)
    ref = oracle.psiN(sysm.tensors[3], 20, 3, sysm.U, sysm.V, sysm.lam, p1_block=20)
    assert rel_fro(one, ref) < TOL and rel_fro(many, ref) < TOL


def test_n60_order3_full_and_order4_slabs(npf):
    sysm = S.config_n60(0, orders=(3, 4))
    with make_plan(npf, sysm, 4, "fp64") as p:
        ref3 = oracle.psiN(sysm.tensors[3], 60, 3, sysm.U, sysm.V, sysm.lam, p1_block=4)
        assert rel_fro(p.term(3), ref3) < TOL
        rng = np.random.default_rng(0)
        for _ in range(3):
            pre = [int(x) for x in rng.integers(0, 60, size=3)]
            ref = oracle.h_slab(sysm.tensors[4], 60, 4, sysm.U, sysm.V, sysm.lam, pre)
            assert rel_fro(p.modal_slab(4, pre), ref) < TOL


def test_collapse_identity_full_size(npf):
    """divide off: Psi_N[i,k] = -(1/N!) sum_j psi_ij A^j_{k..k} (a closed form at n = 60, N = 4)."""
    sysm = S.config_n60(1, orders=(4,))
    n, N = 60, 4
    diag = [S.packed_count(n, N) - S.packed_count(n - k, N) for k in range(n)]  # rank of (k,k,k,k)
    Akk = sysm.tensors[N][:, diag]
    expect = -(sysm.V @ Akk) / math.factorial(N)
    with make_plan(npf, sysm, N, "fp64") as p:
        p.set_option(npf.OPT_DIVIDE, 0)
        assert rel_fro(p.term(N), expect) < TOL


def test_error_codes(npf):
    sysm = S.config_small(0, orders=(2,))
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 3, precision="fp64") as p:
        with pytest.raises(npf.NpfError) as e:
            p.compute(2)
        assert e.value.status == npf.NPF_ERR_MISSING_TENSOR
        with pytest.raises(npf.NpfError) as e:
            p.compute(4)
        assert e.value.status == npf.NPF_ERR_ARG
        p.set_tensor(3, S.random_packed_tensor(10, 3, 1))
        p.compute(3)   # order 2 missing is skipped, order 3 present
    bad = sysm.V.copy()
    bad[0, 0] += 1e-3
    with pytest.raises(npf.NpfError) as e:
        npf.Plan(sysm.lam, sysm.U, bad, 2)
    assert e.value.status == npf.NPF_ERR_NOT_INVERSE
