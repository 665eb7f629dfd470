"""C-ABI library: it builds, loads without a GPU, exports every symbol that
include/ptrace.h declares, and its host-side stencil (Eq. (8)) matches the
oracle.  No compute call is made (there may be no GPU)."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "ptrace.h")).read()
    return sorted(set(re.findall(r"PT_API\s+int\s+(pt_\w+)\s*\(", txt)))


def test_header_and_binding_agree(ptlib):
    assert header_symbols() == ptlib.exported_symbols()


def test_library_exports_every_declared_symbol(ptlib):
    L = ptlib.lib()
    for name in header_symbols():
        assert hasattr(L, name), name
    assert L.pt_version() >= 100


@pytest.mark.parametrize("mu,p_list,k", [(0, [0], 1), (2, [3], 2), (3, [1, 2], 3), (1, [5], 2), (2, [0], 4)])
def test_stencil_matches_oracle(ptlib, mu, p_list, k):
    from oracle.stencil import displaced_stencil
    got = ptlib.stencil(mu, p_list, k)
    want = displaced_stencil(4, mu, p_list, k)
    assert np.array_equal(got, want)


def test_bad_arguments_are_rejected_without_a_gpu(ptlib):
    import ctypes
    L = ptlib.lib()
    n = ctypes.c_int()
    p = (ctypes.c_int * 1)(1)
    assert L.pt_stencil(7, p, 1, 2, None, 0, ctypes.byref(n)) == ptlib.PT_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    L.pt_last_error(buf, 256)
    assert b"pt_stencil" in buf.value


def test_tile_dims_match_oracle_without_a_gpu(ptlib):
    """pt_tile_dims is host-only: Table 2's tiles and ragged lattices agree
    with the oracle's tile policy (Sec. 3.5)."""
    from oracle.tiles import tile_dims
    cases = [([32, 32, 32, 64], 2, [p], k) for p in range(9) for k in range(1, 11)]
    cases += [([24, 24, 24, 48], 2, [8], 2), ([24, 24, 24, 48], 2, [0, 4], 3), ([12, 18, 30, 7], 1, [2], 1),
              ([64, 64, 64, 64], 0, [8], 8), ([5, 5, 5, 5], 3, [1], 4)]
    for dims, mu, p_list, k in cases:
        assert ptlib.tile_dims(dims, mu, p_list, k) == tile_dims(dims, mu, p_list, k), (dims, mu, p_list, k)
    import ctypes
    out = (ctypes.c_int * 4)()
    assert ptlib.lib().pt_tile_dims(ptlib._ints([8, 8, 8, 8]), 4, ptlib._ints([1]), 1, 1, out) == ptlib.PT_ERR_ARG
