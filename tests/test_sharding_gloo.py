"""Multi-rank layout (world size 2, gloo on CPU): ranks take disjoint noise
sets, the timing reduction takes the slowest rank and sums the work, and the
gathered per-set estimates equal those of one rank doing all sets (checked
with the oracle's estimator, which is what each rank's GPU run reproduces)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2106_01275_gb300 import sharding
    import oracle.estimator as OE
    from oracle.colouring import greedy_colour
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    col, m = greedy_colour(dims, 0, [p], 1, 0)
    set0, n = sharding.rank_sets(rank, 3)
    est = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 5, n, 0, 0, [p], 1e-12, set0=set0)
    allest = sharding.gather_estimates(est)
    t, u = sharding.reduce_timing(10.0 + rank, 100 * (rank + 1))
    np.save(os.path.join(out_dir, "r%d.npy" % rank), np.array([set0, n, t, u]))
    np.save(os.path.join(out_dir, "est%d.npy" % rank), allest)
    dist.destroy_process_group()


def test_two_rank_sharding(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert (r0[0], r0[1]) == (0, 3) and (r1[0], r1[1]) == (3, 3)      # disjoint sets 0..2, 3..5
    assert r0[2] == r1[2] == 11.0                                       # slowest rank
    assert r0[3] == r1[3] == 300.0                                      # summed work
    e0 = np.load(tmp_path / "est0.npy")
    e1 = np.load(tmp_path / "est1.npy")
    import oracle.estimator as OE
    from oracle.colouring import greedy_colour
    col, m = greedy_colour([4, 4, 4, 4], 0, [1], 1, 0)
    want = OE.probed_estimates(OE.Laplacian([4, 4, 4, 4], 0.1), col, m, 5, 6, 0, 0, [1], 1e-12)
    assert np.allclose(e0, want, rtol=1e-10) and np.array_equal(e0, e1)
