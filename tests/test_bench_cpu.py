"""Host logic of bench.py (no GPU): the DRAM-traffic record is reported only for the kernel
sources it was captured on, both arms describe the same workload, and the algorithmic work
counts follow their closed forms."""
import json
import os
import shutil
from math import comb

import pytest

import bench


def test_traffic_record_matches_current_sources():
    """The committed record is reported exactly while the kernel sources hash to its build."""
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_split_mode_product_n120.json")))
    current = bench.code_hash([os.path.join(bench.ROOT, s) for s in d["sources"]])
    expect = d["traffic_per_launch"] if current == d["code_sha256"] else None
    assert bench.measured_traffic("split_mode_product", "n120") == expect
    assert d["traffic_per_launch"] == d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]
    assert bench.measured_traffic("split_reduce", "n120") is None      # no record
    assert bench.measured_traffic("split_mode_product", "n60") is None


def test_traffic_record_is_dropped_when_a_source_changes(tmp_path, monkeypatch):
    """A copy of the tree whose kernel code changes reports no traffic; comments and whitespace
    do not count."""
    root = tmp_path / "repo"
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_split_mode_product_n120.json")))
    (root / "profiles").mkdir(parents=True)
    for src in d["sources"]:
        dst = root / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, src), dst)
    d["code_sha256"] = bench.code_hash([str(root / s) for s in d["sources"]])
    with open(root / "profiles" / "dram_split_mode_product_n120.json", "w") as f:
        json.dump(d, f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.measured_traffic("split_mode_product", "n120") == d["traffic_per_launch"]
    with open(root / d["sources"][0], "ab") as f:
        f.write(b"\n// a comment\n/* and a block\n   comment */\n")
    assert bench.measured_traffic("split_mode_product", "n120") == d["traffic_per_launch"]
    with open(root / d["sources"][0], "ab") as f:
        f.write(b"static int unused_marker = 0;\n")
    assert bench.measured_traffic("split_mode_product", "n120") is None


def test_both_arms_share_the_workload_config():
    ours = bench.workload_config(120, (3, 4), "split_bf16")
    ref = bench.workload_config(120, (3, 4), "fp64 (CPU oracle)")
    assert {k: v for k, v in ours.items() if k != "precision"} == \
           {k: v for k, v in ref.items() if k != "precision"}
    assert ours["entries_per_step"] == 120 ** 4 + 120 ** 5


@pytest.mark.parametrize("n", [20, 60, 120])
def test_algorithmic_work_closed_forms(n):
    """Per-order counts of the tensor kernels (order 3 alone: mode products c = 1, 2)."""
    pairs = bench.PAIRS["split_bf16"]
    saved = bench.ORDERS
    try:
        bench.ORDERS = (3,)
        up, _ = bench.algorithmic_work_per_step("split_upper_contraction", n, "split_bf16")
        mp, kind = bench.algorithmic_work_per_step("split_mode_product", n, "split_bf16")
        dv, _ = bench.algorithmic_work_per_step("split_mode_divide", n, "split_bf16")
    finally:
        bench.ORDERS = saved
    assert kind == "flops"
    assert up == comb(n + 2, 3) * n * n * 4 * pairs
    # c = 1: n (i) x n (p) x n^2 (a's) x n (K) x 8; c = 2: n x C(n+1, 2) x n x n x 8
    assert mp == (n * n * n * n * n * 8 + n * comb(n + 1, 2) * n * n * 8) * pairs
    assert dv == n * comb(n + 2, 3) * n * 8 * pairs


@pytest.mark.parametrize("n,N", [(6, 3), (7, 4), (120, 3)])
def test_expansion_bytes_count_gathers_and_rows(n, N):
    """split_expand per upper index: one 32-byte record per (sorted prefix, a_N) gathered, and
    S x 4 bytes per entry of every written row (rows (a_1..a_{N-1}) whose shared a's, all but the
    last, are non-decreasing), counted here by enumeration."""
    import itertools
    saved = bench.ORDERS
    try:
        bench.ORDERS = (N,)
        got, kind = bench.algorithmic_work_per_step("split_expand", n, "split_bf16")
    finally:
        bench.ORDERS = saved
    assert kind == "bytes"
    if n > 10:
        prefixes = comb(n + N - 2, N - 1)
        rows = comb(n + N - 3, N - 2) * n
    else:
        prefixes = sum(1 for _ in itertools.combinations_with_replacement(range(n), N - 1))
        rows = sum(1 for t in itertools.product(range(n), repeat=N - 1)
                   if all(t[m] <= t[m + 1] for m in range(N - 3)))
    assert got == n * (prefixes * n * 32 + rows * n * 4 * 6)
