"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/ttn.h, and host-side validation rejects bad
trees before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_15460_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ttn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttn_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["ttn_create", "ttn_set_sop_hamiltonian", "ttn_step", "ttn_expect",
                     "ttn_step_batch", "ttn_reduced_density", "ttn_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib_path):
    from paper_2503_15460_gb300 import ttn
    assert set(declared_symbols()) <= set(ttn.EXPORTED)


@pytest.mark.parametrize("parent,phys,bond,msg", [
    ([0, 0, 0], [0, 2, 2], [1, 2, 2], "parent[0]"),
    ([-1, 0, 0], [0, 2, 0], [1, 2, 2], "no children"),
    ([-1, 0, 0], [0, 2, 2], [1, 3, 2], "exceeds"),          # leaf bond > d
    ([-1, 0, 0], [0, 2, 4], [1, 2, 4], "exceeds"),          # child bond > product of the others
    ([-1, 2, 0], [0, 2, 2], [1, 2, 2], "parent[1]"),
])
def test_create_rejects_invalid_trees(lib_path, parent, phys, bond, msg):
    from paper_2503_15460_gb300 import ttn
    with pytest.raises(ttn.TTNError) as e:
        ttn.ttn_create(parent, phys, bond, ttn.TTN_FP64)
    assert e.value.status == ttn.TTN_E_INVALID
    assert msg in str(e.value)
