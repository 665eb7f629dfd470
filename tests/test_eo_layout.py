"""Even-odd half-field layout of the library (pt_eo_layout, host only; the
same index functions run in the even-odd kernels) against the oracle's
even / odd split and its neighbour tables.  No GPU needed."""
import os
import shutil

import numpy as np
import pytest

from oracle import evenodd as EO
from oracle import operators as ops


@pytest.fixture(scope="module")
def ptlib():
    from paper_2106_01275_gb300 import build
    if build.needs_build():
        if not shutil.which(build.NVCC) and not os.path.exists(build.NVCC):
            pytest.skip("nvcc not available to build libptrace.so")
        build.build()
    from paper_2106_01275_gb300 import ptrace
    return ptrace


@pytest.mark.parametrize("dims", [[2, 2, 2, 2], [4, 2, 6, 2], [6, 4, 2, 8], [2, 4, 4, 6], [8, 8, 8, 16]])
def test_layout_matches_the_oracle_split(ptlib, dims):
    ev, od = EO.split(dims)
    fwd, bwd = ops.neighbour_tables(dims)
    for parity, mine, other in ((0, ev, od), (1, od, ev)):
        site, nbr = ptlib.eo_layout(dims, parity)
        assert np.array_equal(site, mine)                               # storage order within the parity
        assert np.array_equal(site >> 1, np.arange(site.size))          # entry h holds site 2h or 2h + 1
        for mu in range(4):
            assert np.array_equal(other[nbr[:, 2 * mu]], fwd[mu][mine])  # x + mu, in the other parity
            assert np.array_equal(other[nbr[:, 2 * mu + 1]], bwd[mu][mine])


def test_odd_sides_refused(ptlib):
    with pytest.raises(ptlib.PtraceError):
        ptlib.eo_layout([4, 3, 4, 4], 0)
    with pytest.raises(ptlib.PtraceError):
        ptlib.eo_layout([4, 4, 4, 4], 2)
