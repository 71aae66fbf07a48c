"""The C-ABI library loads without a GPU and exports every function include/npf.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_08968_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(npf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["npf_plan", "npf_set_tensor", "npf_compute", "npf_destroy"]:
        assert required in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), name


def test_host_only_calls_without_gpu(lib):
    import paper_2509_08968_gb300 as npf
    r = npf.alg1_batches(4, 351, 8.0)
    assert r["batches"] == 15
    assert npf.launch_count() >= 0
