"""Tile widths of the row kernel against the CPU oracle, at each row radix.

At 32 complex columns or fewer a one-pass launch (upper contraction, mode products) alternates two
TMEM accumulator sets, tile t on set t mod 2 with its four levels 2 x width columns apart, so the
next tile's MMAs run during the epilogue; at 64 columns the levels fill TMEM and the epilogue runs
in series. Width 48 runs the mode products at radix 128 in 48-column tiles (N = 96, three column
tiles per radix) with two passes over K and the level-3 hold, and 32 elsewhere. The divide and the
reduction (two passes over K with the level-3 hold) run 64 columns wide whatever the width asked
for. Each width at each radix (32 for n <= 32, 64 for n <= 64, else
128), for the FP64-emulating form (6 slices, bar 1e-10) and the FP32 form (4 slices, bar 1e-5),
against the oracle's Psi_3; n = 68 with an odd and an even number of tiles per CTA across the
launches of a term.
"""
import pytest

import npf_synth as S
import oracle
from tests._util import rel_fro

pytestmark = pytest.mark.gpu
TOL = {"split_bf16": 1e-10, "fp32": 1e-5}
_REF = {}


@pytest.fixture(scope="module")
def npf():
    from paper_2509_08968_gb300 import build
    build.build()
    import paper_2509_08968_gb300 as m
    return m


def _system(n):
    sysm = S.near_resonant_system(n, 7000 + n)
    sysm.tensors[3] = S.random_packed_tensor(n, 3, 7000 + 3 * n)
    return sysm


def _ref(n, sysm):
    if n not in _REF:
        _REF[n] = oracle.psiN(sysm.tensors[3], n, 3, sysm.U, sysm.V, sysm.lam, p1_block=8)
    return _REF[n]


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("width", [16, 32, 48, 64])
@pytest.mark.parametrize("n", [30, 60, 68])
def test_tile_width_matches_oracle(npf, n, width, prec):
    sysm = _system(n)
    ref = _ref(n, sysm)
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 3, precision=prec) as p:
        p.set_option(npf.OPT_TILE_N, width)
        p.set_tensor(3, sysm.tensors[3])
        got = p.term(3)
        assert rel_fro(got, ref) < TOL[prec], (n, width, prec, rel_fro(got, ref))
        # the same plan again: a second term reuses the buffers and the tile lists
        assert rel_fro(p.term(3), got) < 1e-13
