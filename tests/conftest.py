import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="module")
def ptlib():
    """The library's binding, built if needed (the host-only entry points need no GPU)."""
    from paper_2106_01275_gb300 import build
    if build.needs_build():
        if not shutil.which(build.NVCC) and not os.path.exists(build.NVCC):
            pytest.skip("nvcc not available to build libptrace.so")
        build.build()
    from paper_2106_01275_gb300 import ptrace
    return ptrace
