"""The allocation-free entry point pt_colour_conflicts_noalloc, called through
the C ABI, against the context-based pt_colour_conflicts.

It serves callers that cannot allocate device memory (their own pool
allocator owns the device, or cudaMalloc's implicit synchronisation is not
acceptable to them).  Its scratch is a static device array shared by every
call, so the test makes two calls in a row and checks that the second does
not see the first one's count.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle.colouring import greedy_colour

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_01275_gb300 import build
    build.build()
    from paper_2106_01275_gb300 import ptrace
    return ptrace


def test_noalloc_conflicts_match_context_version(pt):
    import torch
    ctx = pt.Context(0)
    cases = [([8, 8, 16, 8], 2, [2], 2), ([6, 5, 7, 3], 1, [1, 3], 1)]
    for dims, mu, p, k in cases:
        N = int(np.prod(dims))
        good, _ = greedy_colour(dims, mu, p, k, 0)
        bad = np.zeros(N, dtype=np.int32)                       # one colour: invalid
        half = good.copy()
        half[: N // 2] = 0                                       # partly invalid
        for colv in (bad, good, half, bad):                      # consecutive calls share the scratch
            col = torch.as_tensor(colv).cuda()
            want = pt.conflicts(ctx, dims, mu, p, k, col)
            got = pt.conflicts_noalloc(dims, mu, p, k, col)
            assert got == want
        assert pt.conflicts_noalloc(dims, mu, p, k, torch.as_tensor(good).cuda()) == 0


def test_noalloc_rejects_oversized_stencil(pt):
    import torch
    col = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(pt.PtraceError) as ei:
        pt.conflicts_noalloc([2, 2, 2, 2], 0, [0], 12, col)      # |N(0,0,12)| in 4D exceeds 16384
    assert ei.value.code == pt.PT_ERR_ARG


def test_noalloc_overlapping_displacements_fit(pt):
    """Repeated displacements produce each stencil offset twice: 2 x 11968
    raw rows for (p = 0, k = 11) listed twice, above the 16384-offset limit,
    but 11968 distinct ones, which fit.  The result must equal the context
    version's on an invalid and a partly valid colouring."""
    import torch
    ctx = pt.Context(0)
    dims, mu, k = [6, 5, 7, 4], 3, 11
    assert pt.stencil(mu, [0], k).shape[0] == 11968
    N = int(np.prod(dims))
    rng = np.random.default_rng(7)
    for colv in (np.zeros(N, np.int32), rng.integers(0, N // 2, N).astype(np.int32)):
        col = torch.as_tensor(colv).cuda()
        want = pt.conflicts(ctx, dims, mu, [0], k, col)
        for p in ([0, 0], [0, 0, 0]):
            assert pt.conflicts_noalloc(dims, mu, p, k, col) == want
