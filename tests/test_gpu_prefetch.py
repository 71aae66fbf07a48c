"""Double-buffered tensor upload (npf_compute_prefetch): a call computes with the current tensors
while the next ones upload, and the next tensor-using call computes with those. Checked against
the oracle for both tensor sets, over several ping-pong rounds, from pinned host and device
sources, through npf_batch_compute, and for both precision families."""
import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import make_plan, rel_fro

pytestmark = pytest.mark.gpu

N_STATES = 32


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


@pytest.fixture(scope="module")
def systems():
    """One modal system with two different tensor sets (orders 2 and 3) and the oracle's NPF of
    order 3 for each."""
    a = S.config_blocks(N_STATES, seed=21, orders=(2, 3))
    b = S.config_blocks(N_STATES, seed=22, orders=(2, 3))
    b_on_a = S.ModalSystem(n=a.n, A1=a.A1, lam=a.lam, U=a.U, V=a.V, P=a.P, tensors=dict(b.tensors))
    ref = {"a": oracle.npf_orders(a, 3, p1_block=8), "b": oracle.npf_orders(b_on_a, 3, p1_block=8)}
    return a, b_on_a, ref


@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-10), ("fp64", 1e-12)])
def test_prefetch_ping_pong(npf, systems, prec, tol):
    a, b, ref = systems
    sets = {"a": a.tensors, "b": b.tensors}
    with make_plan(npf, a, 3, prec) as p:
        cur = "a"
        for _ in range(4):
            nxt = "b" if cur == "a" else "a"
            got = p.compute_prefetch(3, next_tensors=sets[nxt])
            assert rel_fro(got, ref[cur]) < tol          # this call: the current tensors
            cur = nxt
        assert rel_fro(p.compute(3), ref[cur]) < tol     # the plain call activates the last ones
        np.testing.assert_array_equal(p.get_tensor(3), sets[cur][3])
        np.testing.assert_array_equal(p.get_tensor(2), sets[cur][2])


def test_prefetch_pinned_and_device_sources(npf, systems):
    import torch
    a, b, ref = systems
    pinned = {N: torch.from_numpy(t).pin_memory() for N, t in b.tensors.items()}
    dev = {N: torch.from_numpy(t).cuda() for N, t in a.tensors.items()}
    out = torch.empty((N_STATES, N_STATES), dtype=torch.complex128).pin_memory()
    with make_plan(npf, a, 3, "split_bf16") as p:
        p.compute_prefetch(3, out, pinned)
        assert rel_fro(out.numpy(), ref["a"]) < 1e-10
        p.compute_prefetch(3, out, dev)
        assert rel_fro(out.numpy(), ref["b"]) < 1e-10
        assert rel_fro(p.compute(3), ref["a"]) < 1e-10


def test_prefetch_one_order_only(npf, systems):
    """Only order 3 prefetched: order 2 keeps its tensor."""
    a, b, ref = systems
    mixed = S.ModalSystem(n=a.n, A1=a.A1, lam=a.lam, U=a.U, V=a.V, P=a.P,
                          tensors={2: a.tensors[2], 3: b.tensors[3]})
    want = oracle.npf_orders(mixed, 3, p1_block=8)
    with make_plan(npf, a, 3, "split_bf16") as p:
        p.compute_prefetch(3, next_tensors={3: b.tensors[3]})
        assert rel_fro(p.compute(3), want) < 1e-10


def test_prefetch_then_batch(npf, systems):
    a, b, ref = systems
    with make_plan(npf, a, 3, "split_bf16") as p, make_plan(npf, a, 3, "split_bf16") as q:
        p.compute_prefetch(3, next_tensors=b.tensors)
        outs = [np.empty((N_STATES, N_STATES), np.complex128) for _ in range(2)]
        npf.batch_compute([p, q], [3, 3], outs)
        assert rel_fro(outs[0], ref["b"]) < 1e-10
        assert rel_fro(outs[1], ref["a"]) < 1e-10


def test_prefetch_bad_arguments(npf, systems):
    a, b, ref = systems
    with make_plan(npf, a, 3, "split_bf16") as p:
        with pytest.raises(npf.NpfError) as e:
            p.compute_prefetch(3, next_tensors={4: b.tensors[3]})     # order above N_max
        assert e.value.status == npf.NPF_ERR_ARG
        # nothing was staged: the plan still computes with its own tensors
        assert rel_fro(p.compute(3), ref["a"]) < 1e-10
