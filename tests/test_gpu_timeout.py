"""The tensor-core pipeline's bounded waits: a test hook withholds the first completion signal,
the epilogue's wait runs out (~2 s), the call reports NPF_ERR_TIMEOUT, and the CUDA context stays
usable (no fault, trap or hang is involved)."""
import time

import pytest

import npf_synth as S
import oracle
from tests._util import make_plan, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


def test_bounded_wait_reports_timeout_and_recovers(npf):
    sysm = S.config_small(0, orders=(2,))
    ref = oracle.psiN(sysm.tensors[2], 10, 2, sysm.U, sysm.V, sysm.lam, p1_block=10)
    with make_plan(npf, sysm, 2, "split_bf16") as p:
        p.set_option(npf.OPT_DEBUG_STALL, 1)
        t0 = time.time()
        with pytest.raises(npf.NpfError) as e:
            p.term(2)
        assert e.value.status == npf.NPF_ERR_TIMEOUT
        assert time.time() - t0 < 60
        p.set_option(npf.OPT_DEBUG_STALL, 0)
        assert rel_fro(p.term(2), ref) < 1e-10
