"""The contraction kernels on A1 as an order-1 tensor: Psi A1 Phi = diag(lambda).

The generator builds A1 = P B P^-1 with U = P W and V = U^-1, so running the chain of Algorithm 2
on the Jacobian (its lower index contracted with Phi, its upper index with Psi, 1/1!) with the
divide off must return the eigenvalues on the diagonal and zeros elsewhere. This checks the
first-contraction, expansion and mode-product GEMMs of every precision form against a closed form
at every row radix (n = 10: 32, n = 40: 64, n = 68 and 120: 128). With the divide on, the diagonal
denominators lambda_i - lambda_i are exactly zero and take the clamp of Algorithm 2 step 9.

The sums cancel: the result diag(lambda) is smaller than the magnitudes that enter it by the
factor kappa = || |Psi| |A1| |Phi| ||_F / ||lambda||_2 (40 at n = 120, 2500 for the dense n = 10
system), so a form with unit error u on full-scale sums shows ~u kappa here. The FP64-emulating
split form and the native FP64 form stay within their usual bars; the FP32 form (4 slices, 32-bit
operands) is held to max(1e-5, 32 * 2^-31 * kappa), its unit error times kappa with a margin.
"""
import numpy as np
import pytest

import npf_synth as S
from tests._util import rel_fro

pytestmark = pytest.mark.gpu
TOL = {"split_bf16": 1e-10, "fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


def _system(n):
    return S.modal_system(n, 5) if n % 4 else S.config_blocks(n, 5, orders=())


def _bar(prec, sysm):
    if prec != "fp32":
        return TOL[prec]
    kappa = (np.linalg.norm(np.abs(sysm.V) @ np.abs(sysm.A1) @ np.abs(sysm.U))
             / np.linalg.norm(sysm.lam))
    return max(TOL[prec], 32 * 2.0 ** -31 * kappa)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "fp64"])
@pytest.mark.parametrize("n", [10, 40, 68, 120])
def test_order1_chain_gives_eigenvalues(npf, n, prec):
    sysm = _system(n)
    bar = _bar(prec, sysm)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 1, precision=prec) as p:
        p.set_tensor(1, np.ascontiguousarray(sysm.A1))
        p.set_option(npf.OPT_DIVIDE, 0)
        got = p.modal_slab(1, [])
        assert rel_fro(got, np.diag(sysm.lam)) < bar, rel_fro(got, np.diag(sysm.lam))
        p.set_option(npf.OPT_DIVIDE, 1)
        eps = 1e-8
        hd = p.modal_slab(1, [])
    # D = lambda_p - lambda_i: the diagonal is clamped to eps, the rest is 0 / D
    assert rel_fro(np.diag(hd), sysm.lam / eps) < bar
    off = hd - np.diag(np.diag(hd))
    assert np.abs(off).max() < bar * np.abs(sysm.lam).max() / eps


def test_order1_term_is_rejected(npf):
    sysm = _system(10)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 1, precision="split_bf16") as p:
        p.set_tensor(1, np.ascontiguousarray(sysm.A1))
        with pytest.raises(npf.NpfError) as e:
            p.term(1)
        assert e.value.status == npf.NPF_ERR_ARG
