"""Batched execution of many independent systems (one recorded CUDA graph) and the tile-width
autotuner, against the CPU oracle.

Workload shape: systems of uneven size n ~ U{20..80} and order N in {2, 3}, eigenvalues with a
harmonic ladder so that about 5% of the ordered mode pairs sit within 1e-3 of a resonance.
"""
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


@pytest.fixture(scope="module")
def systems():
    return S.batch_systems(count=12, seed=5)


@pytest.fixture(scope="module")
def references(systems):
    return [oracle.npf_orders(sysm, N, p1_block=sysm.lam.shape[0]) for sysm, N in systems]


def _kappa(lam, N):
    """max |lambda| over the smallest |lambda_p1 + .. + lambda_pN - lambda_i|."""
    lam = np.asarray(lam)
    sums = lam
    for _ in range(N - 2):
        sums = (sums[..., None] + lam).reshape(-1)
    dmin = np.inf
    for s in np.array_split(sums, max(1, sums.size // 4096)):
        d = np.abs(s[:, None, None] + lam[None, :, None] - lam[None, None, :])
        dmin = min(dmin, float(d.min()))
    return float(np.abs(lam).max()) / dmin


def _plans(npf, systems, precision="split_bf16", tile=0):
    plans = []
    for sysm, N in systems:
        p = make_plan(npf, sysm, N, precision)
        p.set_option(npf.OPT_TILE_N, tile)
        plans.append(p)
    return plans


def test_batch_matches_oracle_and_replays(npf, systems, references):
    plans = _plans(npf, systems)
    orders = [N for _, N in systems]
    try:
        outs = [np.zeros((s.lam.shape[0],) * 2, np.complex128) for s, _ in systems]
        npf.batch_compute(plans, orders, outs)
        for (sysm, N), got, ref in zip(systems, outs, references):
            assert rel_fro(got, ref) < TOL, (sysm.lam.shape[0], N, rel_fro(got, ref))
        # the second call records the graph and replays it, the third replays it: the same
        # numbers up to the order of the FP64 atomic additions of the reduction; kernels are
        # counted per replay
        for _ in range(2):
            c0 = npf.launch_count()
            outs2 = [np.zeros_like(o) for o in outs]
            npf.batch_compute(plans, orders, outs2)
            assert npf.launch_count() > c0
            for a, b in zip(outs, outs2):
                assert rel_fro(b, a) < 1e-13
        # every (n, order) key was tuned to one of the candidate widths
        for sysm, N in systems:
            assert npf.tuned_tile(sysm.lam.shape[0], N) in (16, 32, 48, 64)
    finally:
        for p in plans:
            p.close()


def test_batch_equals_single_calls(npf, systems):
    """With a fixed tile width the batch runs the same kernels as single calls: equal results."""
    plans = _plans(npf, systems[:6], tile=32)
    orders = [N for _, N in systems[:6]]
    try:
        single = [p.compute(N) for p, N in zip(plans, orders)]
        outs = [np.zeros_like(x) for x in single]
        npf.batch_compute(plans, orders, outs)
        for a, b in zip(single, outs):
            assert rel_fro(b, a) < 1e-14
    finally:
        for p in plans:
            p.close()


def test_batch_recaptures_after_a_change(npf, systems, references):
    plans = _plans(npf, systems[:4], tile=64)
    orders = [N for _, N in systems[:4]]
    try:
        outs = [np.zeros((s.lam.shape[0],) * 2, np.complex128) for s, _ in systems[:4]]
        npf.batch_compute(plans, orders, outs)
        npf.batch_compute(plans, orders, outs)   # recorded
        # new tensor values for system 1 (same shape: the recorded graph is replayed and must
        # read the new operands)
        sysm, N = systems[1]
        n = sysm.lam.shape[0]
        t2 = 0.5 * sysm.tensors[N]
        plans[1].set_tensor(N, t2)
        npf.batch_compute(plans, orders, outs)
        half = S.ModalSystem(n=n, A1=sysm.A1, lam=sysm.lam, U=sysm.U, V=sysm.V, P=sysm.P,
                             tensors={N: t2})
        ref_half = oracle.npf_orders(half, N, p1_block=n)
        assert rel_fro(outs[1], ref_half) < TOL
        for b in (0, 2, 3):
            assert rel_fro(outs[b], references[b]) < TOL
    finally:
        for p in plans:
            p.close()


def test_batch_fp64_and_mixed_orders(npf, systems, references):
    plans = _plans(npf, systems[:5], precision="fp64")
    orders = [N for _, N in systems[:5]]
    orders[0] = 1   # linear participation factors only
    try:
        outs = [np.zeros((s.lam.shape[0],) * 2, np.complex128) for s, _ in systems[:5]]
        npf.batch_compute(plans, orders, outs)
        sysm0 = systems[0][0]
        np.testing.assert_allclose(outs[0], sysm0.U * sysm0.V.T, rtol=0, atol=1e-14)
        # native FP64 against the oracle: both round the resonance denominator
        # lambda_p1 + .. + lambda_pN - lambda_i (|lambda| up to ~15) in their own order, and this
        # workload places some denominators near 1e-4, so the result is only fixed to about
        # eps * max|lambda| / min|D| (relative); the bar is a small multiple of that
        for b in range(1, 5):
            sysm, N = systems[b]
            tol = max(1e-12, 8 * np.finfo(float).eps * _kappa(sysm.lam, N))
            assert rel_fro(outs[b], references[b]) < tol, (b, tol)
    finally:
        for p in plans:
            p.close()


def test_batch_rejects_bad_arguments(npf, systems):
    plans = _plans(npf, systems[:2])
    try:
        outs = [np.zeros((s.lam.shape[0],) * 2, np.complex128) for s, _ in systems[:2]]
        with pytest.raises(npf.NpfError):
            npf.batch_compute([plans[0], plans[0]], [2, 2], [outs[0], outs[0]])
        with pytest.raises(npf.NpfError):
            npf.batch_compute(plans, [9, 2], outs)
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("tile", [16, 32])
def test_tile_widths(npf, tile):
    sysm = S.config_blocks(60, seed=4, orders=(3,))
    with make_plan(npf, sysm, 3, "split_bf16") as p:
        p.set_option(npf.OPT_TILE_N, tile)
        ref = oracle.psiN(sysm.tensors[3], 60, 3, sysm.U, sysm.V, sysm.lam, p1_block=60)
        assert rel_fro(p.term(3), ref) < TOL


@pytest.mark.parametrize("prec,tol", [("split_bf16", TOL), ("fp64", 1e-12)])
def test_set_modes_replaces_the_system(npf, prec, tol):
    s1 = S.config_blocks(40, seed=1, orders=(3,))
    s2 = S.config_blocks(40, seed=2, orders=(3,))
    with make_plan(npf, s1, 3, prec) as p:
        p.compute(3)
        p.set_modes(s2.lam, s2.U, s2.V)
        mixed = S.ModalSystem(n=40, A1=s2.A1, lam=s2.lam, U=s2.U, V=s2.V, P=s2.P,
                              tensors=dict(s1.tensors))
        ref = oracle.npf_orders(mixed, 3, p1_block=40)
        assert rel_fro(p.compute(3), ref) < tol
        with pytest.raises(npf.NpfError):
            p.set_modes(s2.lam, s2.U, 2.0 * s2.V)   # V is no longer U^-1
