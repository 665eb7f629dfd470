"""Resumable trace estimation: per-set estimates logged and resumed after an
interruption raised on the host, extended to more sets, a line cut short by
a crash dropped, damage and foreign logs refused.  The solves come from the
oracle behind a fake binding (no GPU needed); the resumed estimates equal an
uninterrupted run bit for bit."""
import types

import numpy as np
import pytest

import oracle.estimator as OE
from oracle.colouring import greedy_colour
from paper_2106_01275_gb300 import checkpoint as ck
from paper_2106_01275_gb300 import ptrace as pt

DIMS, M2, MU, PS = [4, 4, 4, 4], 0.1, 0, [0, 1, 2]


@pytest.fixture()
def setup(monkeypatch):
    col, m = greedy_colour(DIMS, MU, PS, 1, 0)
    calls = []
    state = {"fail_at": None}

    def trace(op, c, n_colours, mu, p_list, noise, seed, set0, n_sets, dilute, prec, tol, maxit):
        calls.append((set0, n_sets))
        if state["fail_at"] is not None and len(calls) == state["fail_at"]:
            raise RuntimeError("injected failure")
        est = OE.probed_estimates(OE.Laplacian(DIMS, M2), c, n_colours, seed, n_sets, 0, mu, p_list, 1e-12,
                                  set0=set0)
        return est, None, None, {}

    monkeypatch.setattr(pt, "trace", trace)
    op = types.SimpleNamespace(dims=DIMS, dof=1, m2=M2)
    want = OE.probed_estimates(OE.Laplacian(DIMS, M2), col, m, 7, 5, 0, MU, PS, 1e-12)
    return op, col, m, calls, state, want


def _run(op, col, m, path, n_sets, chunk=2, seed=7):
    return ck.trace_resumable(op, col, m, MU, PS, "z2", seed, n_sets, str(path), chunk=chunk)


def test_uninterrupted_and_extended(setup, tmp_path):
    op, col, m, calls, state, want = setup
    log = tmp_path / "run.jsonl"
    est = _run(op, col, m, log, 3)
    assert np.array_equal(est, want[:3]) and calls == [(0, 2), (2, 1)]
    est = _run(op, col, m, log, 5)                       # two more sets, nothing recomputed
    assert np.array_equal(est, want) and calls[2:] == [(3, 2)]
    assert np.array_equal(_run(op, col, m, log, 4), want[:4]) and len(calls) == 3


def test_resume_after_an_interruption(setup, tmp_path):
    op, col, m, calls, state, want = setup
    log = tmp_path / "run.jsonl"
    state["fail_at"] = 2
    with pytest.raises(RuntimeError, match="injected"):
        _run(op, col, m, log, 5)
    assert np.array_equal(ck.read_log(str(log), ck.run_key(op, col, MU, PS, "z2", 7, True, "mixed_fp32", 1e-10)),
                          want[:2])
    state["fail_at"] = None
    est = _run(op, col, m, log, 5)
    assert np.array_equal(est, want) and calls[2:] == [(2, 2), (4, 1)]


def test_cut_line_is_dropped_and_damage_refused(setup, tmp_path):
    op, col, m, calls, state, want = setup
    log = tmp_path / "run.jsonl"
    _run(op, col, m, log, 2)
    with open(log, "a") as f:
        f.write('{"set": 2, "est": [[1.5, 0')            # a crash in the middle of a line
    est = _run(op, col, m, log, 3)
    assert np.array_equal(est, want[:3]) and calls[-1] == (2, 1)
    text = open(log).read()
    assert text.endswith("\n") and text.count("\n") == 4  # header + 3 sets
    lines = text.split("\n")
    lines[2] = lines[2].replace('"set": 1', '"set": 9')
    open(log, "w").write("\n".join(lines))
    with pytest.raises(ck.CheckpointError, match="expected set 1"):
        _run(op, col, m, log, 3)
    lines[2] = "not json"
    open(log, "w").write("\n".join(lines))
    with pytest.raises(ck.CheckpointError, match="damaged line"):
        _run(op, col, m, log, 3)


def test_foreign_log_refused_and_cut_header_restarts(setup, tmp_path):
    op, col, m, calls, state, want = setup
    log = tmp_path / "run.jsonl"
    _run(op, col, m, log, 1)
    with pytest.raises(ck.CheckpointError, match="another run"):
        _run(op, col, m, log, 2, seed=8)                 # other noise seed
    other = col.copy()
    other[0] = (other[0] + 1) % m
    with pytest.raises(ck.CheckpointError, match="another run"):
        _run(op, other, m, log, 2)                       # other colouring
    log2 = tmp_path / "cut.jsonl"
    log2.write_text('{"version": 1, "ke')               # header cut short: start afresh
    assert np.array_equal(_run(op, col, m, log2, 2), want[:2])
