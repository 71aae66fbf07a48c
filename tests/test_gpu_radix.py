"""Row radix matched to n on the tensor-core path: 32 for n <= 32, 64 for n <= 64, else 128, so a
128-row tile holds four, two or one operand rows. Systems on both sides of each boundary, for
orders 2 (whose tiles can span several upper indices, the last one padded past the batch), 3 and
4, against the oracle; and a multi-batch run, whose upper-index batches end inside a tile."""
import numpy as np
import pytest

import npf_synth as S
import oracle
from tests._util import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


def _system(n, N, seed):
    sysm = S.near_resonant_system(n, seed)
    sysm.tensors[N] = S.random_packed_tensor(n, N, seed * 7 + N)
    return sysm


@pytest.mark.parametrize("n,N", [(10, 2), (30, 2), (34, 2), (64, 2), (66, 2),
                                 (10, 3), (34, 3), (12, 4)])
def test_radix_boundaries_match_oracle(npf, n, N):
    sysm = _system(n, N, 1000 + n)
    ref = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=8)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N) as p:
        p.set_tensor(N, sysm.tensors[N])
        assert rel_fro(p.term(N), ref) < 1e-10


@pytest.mark.parametrize("n,N", [(30, 2), (34, 3)])
def test_radix_multi_batch(npf, n, N):
    """A memory budget of a few upper indices per batch: batches of 3 or 5 upper indices end
    inside a 128-row tile at radix 32 / 64."""
    sysm = _system(n, N, 2000 + n)
    ref = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=8)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N) as p:
        p.set_tensor(N, sysm.tensors[N])
        full = p.term(N)
        from math import comb
        rad = 32 if n <= 32 else 64
        per_i = 2 * (rad ** (N - 1) * 2 * rad * 2 * 6 + rad ** (N - 1) * 4) + 4096
        fixed = n * (-(-comb(n + N - 1, N) // 128) * 128) * 16 + n * comb(n + N - 1, N) * 32
        p.set_option(npf.OPT_MEM_BUDGET, fixed + 3 * per_i + 8 * 256 + 1024)
        small = p.term(N)
    assert rel_fro(full, ref) < 1e-10
    assert rel_fro(small, ref) < 1e-10


def test_autotuned_plan_term_and_slab(npf):
    """Tile width left to the autotuner (0): the term is tuned, a modal slab runs untuned."""
    n, N = 34, 3
    sysm = _system(n, N, 3000 + n)
    ref = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=8)
    pre = [3, 17]
    ref_slab = oracle.h_slab(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, pre)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N) as p:
        p.set_option(npf.OPT_TILE_N, 0)
        p.set_tensor(N, sysm.tensors[N])
        assert rel_fro(p.modal_slab(N, pre), ref_slab) < 1e-10
        assert rel_fro(p.term(N), ref) < 1e-10


@pytest.mark.parametrize("n,N", [(2, 2), (2, 3), (4, 4), (128, 2)])
def test_smallest_and_largest_systems(npf, n, N):
    """n = 2 and 4 (one mostly padded sub-block) and n = 128, the largest system of the
    tensor-core path (K' = 256: every chunk full, |L0| may reach 2^22)."""
    sysm = _system(n, N, 5000 + n)
    ref = oracle.psiN(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, p1_block=8)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N) as p:
        p.set_tensor(N, sysm.tensors[N])
        assert rel_fro(p.term(N), ref) < 1e-10


def test_n128_order3_slabs(npf):
    n, N = 128, 3
    sysm = _system(n, N, 6000)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, N) as p:
        p.set_tensor(N, sysm.tensors[N])
        for pre in ([5, 127],):   # one prefix: the oracle's slab contracts the whole tensor
            ref = oracle.h_slab(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, pre)
            assert rel_fro(p.modal_slab(N, pre), ref) < 1e-10
