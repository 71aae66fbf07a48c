"""Critical-mode subsets (npf_set_mode_subset) on the tensor-core path against the oracle."""
import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import make_plan, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


@pytest.mark.parametrize("n,N,m", [(10, 3, 4), (60, 3, 20), (20, 4, 7)])
def test_subset_term_and_npf(npf, n, N, m):
    sysm = S.config_blocks(n, seed=n + N, orders=(N,)) if n % 4 == 0 else S.config_small(1, orders=(N,))
    modes = np.random.default_rng(n * 10 + N).choice(n, m, replace=False)   # scrambled order
    ref = oracle.psiN_subset(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, modes)
    with make_plan(npf, sysm, N, "split_bf16") as p:
        p.set_mode_subset(modes)
        got = p.term(N)
        assert rel_fro(got, ref) < TOL, rel_fro(got, ref)
        others = np.setdiff1d(np.arange(n), modes)
        assert np.all(got[others] == 0)
        npf_ref = oracle.npf(sysm.U, sysm.V, ref)
        assert rel_fro(p.compute(N), npf_ref) < TOL
        # back to every mode
        p.set_mode_subset(None)
        full = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=n)
        assert rel_fro(p.term(N), full) < TOL


def test_subset_of_all_modes_in_any_order(npf):
    sysm = S.config_small(2, orders=(3,))
    perm = np.random.default_rng(3).permutation(10)
    full = oracle.psiN(sysm.tensors[3], 10, 3, sysm.U, sysm.V, sysm.lam, p1_block=10)
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        p.set_mode_subset(perm)       # all modes, permuted internally: same results
        assert rel_fro(p.term(3), full) < TOL
        p.set_mode_subset(perm[:9])
        assert rel_fro(p.term(3), oracle.psiN_subset(sysm.tensors[3], 10, 3, sysm.U, sysm.V,
                                                     sysm.lam, perm[:9])) < TOL


def test_subset_rejections(npf):
    sysm = S.config_small(0, orders=(3,))
    with make_plan(npf, sysm, 3, "fp64") as p:
        p.set_mode_subset([0, 1, 2])
        with pytest.raises(npf.NpfError):
            p.term(3)
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        with pytest.raises(npf.NpfError):
            p.set_mode_subset([1, 1])
        p.set_mode_subset([0, 5])
        with pytest.raises(npf.NpfError):
            p.modal_slab(3, [0, 5])
