"""Row ranges of Psi_N (npf_get_term_rows) on the GPU: parity with the oracle's rows, ranges that
add up to the whole term, and a checkpointed computation interrupted and resumed."""
import numpy as np
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


@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-10), ("fp64", 1e-12)])
def test_rows_match_oracle_and_add_up(npf, prec, tol):
    sysm = S.config_blocks(40, seed=9, orders=(3,))
    full = oracle.psiN(sysm.tensors[3], 40, 3, sysm.U, sysm.V, sysm.lam, p1_block=8)
    with make_plan(npf, sysm, 3, prec) as p:
        acc = np.zeros_like(full)
        for lo, hi in ((0, 7), (7, 23), (23, 40)):
            part = p.term_rows(3, lo, hi)
            assert np.all(part[:lo] == 0) and np.all(part[hi:] == 0)
            assert rel_fro(part[lo:hi], full[lo:hi]) < tol
            acc += part
        assert rel_fro(acc, full) < tol
        assert rel_fro(p.term(3), full) < tol


def test_checkpointed_term_resumes(npf, tmp_path):
    from paper_2509_08968_gb300 import shard
    sysm = S.config_blocks(40, seed=10, orders=(3,))
    full = oracle.psiN(sysm.tensors[3], 40, 3, sysm.U, sysm.V, sysm.lam, p1_block=8)
    path = str(tmp_path / "ckpt.npz")
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        with pytest.raises(shard.Interrupted):
            shard.checkpointed_term(p, 3, path, chunk_rows=12, stop_after=2)
        got = shard.checkpointed_term(p, 3, path, chunk_rows=12)
    assert rel_fro(got, full) < 1e-10
