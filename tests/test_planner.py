"""Algorithm 1 batch sizing (host-only arithmetic in libnpf.so) against Tables II and III."""
import json
import os

import pytest

import paper_2509_08968_gb300 as npf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "alg1_tables.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2509_08968_gb300 import build
    build.build()


def _sig(x, digits):
    from math import floor, log10
    return round(x, -int(floor(log10(abs(x)))) + digits - 1)


@pytest.mark.parametrize("case", json.load(open(GOLD))["cases"],
                         ids=lambda c: f"{c['system']}-N{c['order']}")
def test_tables_II_III(case):
    g = json.load(open(GOLD))
    r = npf.alg1_batches(case["n_dim"], case["states"], g["limit_gb"], g["bytes"])
    assert r["BC"] == case["batch_count"]
    assert r["max_batch"] == case["max_batch"]
    if isinstance(case["batches"], float):
        assert _sig(r["batches"], 3) == case["batches"]
    else:
        assert r["batches"] == case["batches"]
    # the tables print totals with 2 decimals or 3 significant digits
    tot = case["total_gb"]
    if case.get("total_printed_sig"):
        assert _sig(r["total_gb"], case["total_printed_sig"]) == tot
    elif tot >= 1e4:
        assert round(r["total_gb"]) == tot
    else:
        assert round(r["total_gb"], 2) == tot
    assert round(r["per_batch_gb"], 2) == case["per_batch_gb"]


def test_degenerate_cases():
    # fits without batching
    r = npf.alg1_batches(3, 10, 8.0)
    assert r["BC"] == [1, 1, 1] and r["batches"] == 1
    # a single element larger than the limit batches every dimension
    r = npf.alg1_batches(2, 4, 1e-12)
    assert r["BC"] == [4, 4] and r["batches"] == 16
    with pytest.raises(npf.NpfError):
        npf.alg1_batches(0, 10, 8.0)
