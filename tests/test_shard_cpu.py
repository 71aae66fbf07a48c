"""Host logic of the row-sharded and resumable terms (paper_2509_08968_gb300/shard.py) on the CPU:
the row ranges, the checkpoint/resume cycle and a two-rank gloo split, with the oracle standing in
for a plan's rows."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import npf_synth as S
import oracle
from paper_2509_08968_gb300 import shard


class OraclePlan:
    """term_rows of one system from the oracle (rows outside the range zero)."""

    def __init__(self, seed=0):
        self.sysm = S.config_small(seed, orders=(3,))
        self.n = 10
        self.full = oracle.psiN(self.sysm.tensors[3], 10, 3, self.sysm.U, self.sysm.V,
                                self.sysm.lam, p1_block=10)
        self.calls = []

    def term_rows(self, order, lo, hi, out=None):
        self.calls.append((lo, hi))
        rows = np.zeros_like(self.full)
        rows[lo:hi] = self.full[lo:hi]
        if out is not None:
            out.copy_(__import__("torch").from_numpy(rows))
            return out
        return rows

    def finish_terms(self, terms, out=None):
        S = np.asarray(terms).reshape(-1, self.n, self.n).sum(axis=0)
        return oracle.npf(self.sysm.U, self.sysm.V, S)


def test_row_ranges():
    for n, parts in ((10, 3), (120, 7), (5, 8)):
        r = shard.row_ranges(n, parts)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == parts
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [hi - lo for lo, hi in r]
        assert max(sizes) - min(sizes) <= 1


def test_checkpoint_resume(tmp_path):
    plan = OraclePlan()
    path = str(tmp_path / "psi3.npz")
    with pytest.raises(shard.Interrupted):
        shard.checkpointed_term(plan, 3, path, chunk_rows=3, stop_after=2)
    assert plan.calls == [(0, 3), (3, 6)]
    with np.load(path) as f:
        assert f["done"].tolist() == [True, True, False, False]
    got = shard.checkpointed_term(plan, 3, path, chunk_rows=3)
    assert plan.calls[2:] == [(6, 9), (9, 10)]          # resumed, no chunk recomputed
    np.testing.assert_array_equal(got, plan.full)
    with pytest.raises(ValueError):
        shard.checkpointed_term(plan, 3, path, chunk_rows=4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2509_08968_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = OraclePlan()
        q.put((rank, sh.term_sharded(plan, 3, dist), plan.calls))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_rows():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (t, c)) for r, t, c in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = OraclePlan().full
    assert got[0][1] == [(0, 5)] and got[1][1] == [(5, 10)]
    for r in range(2):
        np.testing.assert_array_equal(got[r][0], full)   # disjoint rows: the sum is exact


def _rank_npf(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2509_08968_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = OraclePlan()
        q.put((rank, sh.sharded_npf(plan, (3,), dist), plan.calls))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_npf():
    """The row-sharded NPF of the multi-GPU benchmark: each rank forms half the rows, one sum,
    and every rank's NPF equals the single-process one."""
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_npf, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (t, c)) for r, t, c in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    plan = OraclePlan()
    ref = oracle.npf(plan.sysm.U, plan.sysm.V, plan.full)
    assert got[0][1] == [(0, 5)] and got[1][1] == [(5, 10)]
    for r in range(2):
        np.testing.assert_array_equal(got[r][0], ref)
