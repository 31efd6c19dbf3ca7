"""The C ABI library builds, loads without a GPU and exports every entry
point that include/nn.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nn_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04689_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("nn_create", "nn_destroy", "nn_query", "nn_neighbor_nodes", "nn_neighbor_elements",
              "nn_neighbors_both", "nn_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings(lib):
    lib.nn_status_str.restype = ctypes.c_char_p
    assert lib.nn_status_str(0) == b"ok"
    assert b"range" in lib.nn_status_str(4)


def test_binding_mirrors_abi_names():
    from paper_1604_04689_gb300 import nn
    for n in declared_functions():
        assert hasattr(nn, n), n
