"""Mode-interaction NPFs (Eqs. 6-9, npf_interaction) on the GPU against the oracle."""
import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import make_plan, rel_fro

pytestmark = pytest.mark.gpu
TOL = {"split_bf16": 1e-10, "fp64": 1e-12}


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


@pytest.mark.parametrize("prec", ["split_bf16", "fp64"])
@pytest.mark.parametrize("delta", [0.05, 1.0])
def test_small_system(npf, prec, delta):
    sysm = S.config_small(2, orders=(2, 3))
    ref = oracle.interaction_npfs(sysm, 3, delta)
    with make_plan(npf, sysm, 3, prec) as p:
        got = p.interaction(3, delta)
    for M in range(3):
        assert rel_fro(got[M], ref[M]) < TOL[prec], (M, rel_fro(got[M], ref[M]))


def test_n60_order3_split(npf):
    sysm = S.config_n60(1, orders=(2, 3))
    ref = oracle.interaction_npfs(sysm, 3, 0.1, p1_block=6)
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        got = p.interaction(3, 0.1)
    for M in range(3):
        assert rel_fro(got[M], ref[M]) < TOL["split_bf16"], (M, rel_fro(got[M], ref[M]))


def test_missing_order_is_zero(npf):
    sysm = S.config_small(0, orders=(3,))
    ref = oracle.interaction_npfs(sysm, 3, 0.2)
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        got = p.interaction(3, 0.2)
    assert np.all(got[1] == 0)
    assert rel_fro(got[2], ref[2]) < 1e-10 and rel_fro(got[0], ref[0]) < 1e-10
