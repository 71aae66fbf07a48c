"""The swing-model tensors generated on the GPU (npf_set_tensor_swing) against the oracle's
closed form, and NPFs of a swing system computed from them against the oracle."""
import numpy as np
import pytest

import npf_synth as S
import oracle
from oracle import swing
from tests._util import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


@pytest.mark.parametrize("m", [3, 7])
def test_generated_tensor_matches_closed_form(npf, m):
    mod = S.swing_model(m, m)
    sysm = S.swing_system(mod)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 4, precision="split_bf16") as p:
        for N in (2, 3, 4):
            p.set_tensor_swing(N, mod)
            got = p.get_tensor(N)
            ref = swing.packed_tensor(mod, N)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), N


@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-10), ("fp64", 1e-11)])
def test_swing_npf_end_to_end(npf, prec, tol):
    mod = S.swing_model(10, 4)
    sysm = S.swing_system(mod)
    for N in (2, 3):
        sysm.tensors[N] = swing.packed_tensor(mod, N)
    ref = oracle.npf_orders(sysm, 3, p1_block=20)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 3, precision=prec) as p:
        for N in (2, 3):
            p.set_tensor_swing(N, mod)
        assert rel_fro(p.compute(3), ref) < tol
