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


def _bench_worker(rank, world, port, out_dir):
    """One rank of `bench.py --workload lap16 --case small --no-tune` on the
    CPU: gloo instead of NCCL (no GPU visible), the binding's calls stood in
    for by fakes that record which noise sets they were asked for and return
    fixed statistics; rank 1 is slower.  Only the bench's own multi-rank code
    runs: the rank split, the barriers and the max / sum reductions."""
    import sys
    import time
    import types
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.stdout = open(os.path.join(out_dir, "out%d.txt" % rank), "w")
    import torch as T
    import bench
    from paper_2106_01275_gb300 import ptrace as pt

    class Event:
        def __init__(self, **k):
            self.t = None

        def record(self):
            self.t = time.perf_counter()

        def elapsed_time(self, other):
            return (other.t - self.t) * 1e3

    T.cuda.set_device = lambda *a: None
    T.cuda.synchronize = lambda *a: None
    T.cuda.Event = Event
    calls = []

    class Ctx:
        def __init__(self, dev):
            self.device = dev

        def set_memory_budget(self, n):
            pass

        def set_max_slots(self, n):
            pass

        def profile(self, on=True):
            pass

        def profile_read(self, which=0, reset=True):
            return 0, 0.0

    def colour(ctx, dims, mu, ps, k, order):
        return T.zeros(int(np.prod(dims)), dtype=T.int32), 3

    def trace_multi(op, cols, m, mu, ps, noise, seed, set0, n_sets, dilute, prec, tol, maxit):
        calls.append((set0, n_sets))
        time.sleep(0.2 + 0.4 * rank)
        n_rhs = n_sets * sum(m)
        est = np.zeros((len(m), n_sets, len(ps)), dtype=np.complex128)
        est += (set0 + np.arange(n_sets))[None, :, None]
        st = {"n_rhs": n_rhs, "inner_iters": 10 * n_rhs, "outer_iters": 2 * n_rhs,
              "site_rhs_applies": 10 * n_rhs * 65536, "kernel_launches": 7, "n_slots": n_rhs,
              "max_relres": 1e-11, "n_noconv": 0}
        return est, st

    real_empty = T.empty
    T.empty = lambda *a, **k: real_empty(*a, **{kk: v for kk, v in k.items() if kk != "device"})
    pt.Context = Ctx
    pt.laplacian = lambda ctx, dims, m2: types.SimpleNamespace(dims=dims)
    pt.colour = colour
    pt.get_tuning = lambda op, prec: {"delta": 1e-5, "group": 1, "graph_iters": 8, "rhs_block": 1, "overlap": 0,
                                      "evenodd": 1, "seconds_per_rhs": 0.0}
    pt.trace_multi = trace_multi
    sys.argv = ["bench.py", "--case", "small", "--steps", "2", "--warmup", "1", "--no-tune"]
    bench.main()
    sys.stdout.flush()
    np.save(os.path.join(out_dir, "calls%d.npy" % rank), np.array(calls))


def test_bench_multi_rank_path_on_gloo(tmp_path):
    """bench.py's own multi-rank path on two gloo ranks: each rank traces its
    own noise sets (rank r: sets [2r, 2r + 2) of the small workload), rank 0
    alone prints the one JSON line, ms_per_step is the slower rank's and the
    value sums both ranks' site*RHS."""
    import json
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_bench_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    c0 = np.load(tmp_path / "calls0.npy")
    c1 = np.load(tmp_path / "calls1.npy")
    assert {tuple(c) for c in c0} == {(0, 2)} and {tuple(c) for c in c1} == {(2, 2)}
    assert len(c0) == len(c1) == 3                                   # one warm-up + two timed steps
    lines0 = [l for l in open(tmp_path / "out0.txt").read().splitlines() if l.startswith("{")]
    lines1 = [l for l in open(tmp_path / "out1.txt").read().splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and lines1 == []
    d = json.loads(lines0[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak" and d["steps"] == 2
    assert d["ms_per_step"] >= 590.0                                 # rank 1 sleeps 0.6 s per step
    site_both = 2 * 2 * (10 * 2 * 3 * 65536)                         # ranks x steps x site*RHS per step
    assert abs(d["value"] - site_both / (d["ms_per_step"] * 2 / 1e3)) < 1e-6 * d["value"]
    assert d["cpu_baseline"] is None
