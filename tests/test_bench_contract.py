"""The benchmark's reference arm (the FP64 CPU oracle, no GPU needed) prints
the one JSON line the measurement contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "site*RHS/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("lap16")


def test_clock_sampler_reads_reasons():
    """The clocks object of the bench line: median SM clock under load, the
    maximum, and every throttle reason seen active."""
    sys.path.insert(0, ROOT)
    import bench

    class Fake:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                    "0, 2070, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                    "0, 1980, 2070, 1395.2, 0x4, Not Active, Not Active, Not Active, Active"]
            return "\n".join(rows) + "\n", ""

    cs = bench.ClockSampler(0)
    cs.proc = Fake()
    c = cs.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    cs.proc = None
    assert cs.stop()["reasons"] == ["unsampled"]


def test_deflation_leg_json_line(monkeypatch, capsys):
    """`bench.py --workload deflation --case small` end to end on the CPU, with
    every call of the binding stood in for by the oracle (colouring, block
    Lanczos triplets, probed estimates, deflation corrections): one JSON line
    whose checks hold and whose deflated variance is below the plain one."""
    import numpy as np
    import torch
    import types
    sys.path.insert(0, ROOT)
    import bench
    import oracle.estimator as OE
    from oracle import deflation as D
    from oracle.colouring import greedy_colour
    from paper_2106_01275_gb300 import ptrace as pt

    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(pt, "Context", lambda dev: types.SimpleNamespace(device=dev))
    monkeypatch.setattr(pt, "laplacian", lambda ctx, dims, m2: types.SimpleNamespace(dims=dims, m2=m2))
    monkeypatch.setattr(pt, "colour", lambda ctx, dims, mu, ps, k, order: greedy_colour(dims, mu, ps, k, 0))

    def triplets(op, n_ev, block, n_iter, start):
        o = OE.Laplacian(op.dims, op.m2)
        w, V = D.lanczos_lowest(lambda x: np.asarray(o.apply(x)).reshape(-1), o_n(op), n_ev, n_iter, 0,
                                np.float64, block)
        Vt = V.T.reshape(n_ev, -1, 1).astype(np.complex128)
        return Vt, w, Vt

    def o_n(op):
        return int(np.prod(op.dims))

    def trace(op, col, m, mu, ps, noise, seed, set0, n_sets, dil, prec, tol, maxit):
        est = OE.probed_estimates(OE.Laplacian(op.dims, op.m2), col, m, seed, n_sets, 0, mu, ps, 1e-10)
        return est, None, None, {"n_rhs": m * n_sets}

    def terms(op, col, m, mu, ps, noise, seed, set0, n_sets, U, V, M):
        Uh = np.asarray(U).reshape(U.shape[0], -1).T
        Vh = np.asarray(V).reshape(V.shape[0], -1).T
        return (D.deflation_corrections(col, m, seed, n_sets, 0, op.dims, mu, ps, Uh, Vh, M),
                D.deflated_part(Uh, Vh, M, op.dims, mu, ps))

    monkeypatch.setattr(pt, "singular_triplets", triplets)
    monkeypatch.setattr(pt, "trace", trace)
    monkeypatch.setattr(pt, "deflation_terms", terms)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "deflation", "--case", "small"])
    bench.main()
    lines = [l for l in capsys.readouterr().out.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "higher_is_better", "config", "var_plain", "var_deflated", "seconds",
                "check_ritz_vs_closed_form_max_rel", "check_p0_trace_minus_sum_inv_s"):
        assert key in d, key
    assert d["config"]["workload"].startswith("deflation: 8^4")
    assert d["check_ritz_vs_closed_form_max_rel"] < 1e-6 and d["check_p0_trace_minus_sum_inv_s"] < 1e-9
    assert len(d["var_plain"]) == 5 and all(a > 10 * b for a, b in zip(d["var_plain"], d["var_deflated"]))


def test_evenodd_leg_json_line(monkeypatch, capsys):
    """`bench.py --workload evenodd --case small` end to end on the CPU: the
    full-system solves and trace estimates come from the oracle, the even-odd
    ones from the library's host twins of pt_eo_solve and pt_trace_PAinv_eo;
    the line reports fewer even-odd iterations and agreeing solutions and
    estimates."""
    import numpy as np
    import torch
    import types
    sys.path.insert(0, ROOT)
    import bench
    import oracle.estimator as OE
    from paper_2106_01275_gb300 import ptrace as pt

    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(pt, "Context", lambda dev: types.SimpleNamespace(device=dev, set_max_slots=lambda n: None))
    monkeypatch.setattr(pt, "laplacian", lambda ctx, dims, m2: types.SimpleNamespace(kind=0, dims=dims, m2=m2))
    monkeypatch.setattr(pt, "wilson", lambda ctx, dims, U, kappa, ap: types.SimpleNamespace(
        kind=1, dims=dims, U=np.asarray(U), kappa=kappa))

    def oracle_op(op):
        return OE.Laplacian(op.dims, op.m2) if op.kind == 0 else OE.Wilson(op.dims, op.U, op.kappa)

    def solve(op, b, prec, tol, maxit):
        bn = b.numpy()
        xs, its = [], []
        for r in range(bn.shape[0]):
            x, it, _ = oracle_op(op).solve(bn[r], tol)
            xs.append(np.asarray(x).reshape(bn.shape[1:]))
            its.append(it)
        return torch.as_tensor(np.stack(xs)), np.array(its), None, {}

    def eo_solve(op, b, tol, maxit):
        kw = dict(m2=op.m2) if op.kind == 0 else dict(kappa=op.kappa, U=op.U)
        x, its, rel = pt.eo_solve_host(op.kind, op.dims, b.numpy(), tol=tol, maxit=maxit, **kw)
        return torch.as_tensor(x), its, rel

    from oracle.colouring import greedy_colour

    def trace(op, col, m, mu, ps, noise, seed, set0, n_sets, dilute, prec, tol, maxit):
        est = OE.probed_estimates(OE.Laplacian(op.dims, op.m2), col, m, seed, n_sets, 0, mu, ps, 1e-12, set0=set0)
        return est, None, None, {"inner_iters": 0}

    def trace_eo(op, col, m, mu, ps, noise, seed, set0, n_sets, tol, maxit, delta):
        return pt.trace_eo_host(op.dims, op.m2, col, m, mu, ps, noise, seed, set0, n_sets, tol, maxit, delta)

    monkeypatch.setattr(pt, "solve", solve)
    monkeypatch.setattr(pt, "eo_solve", eo_solve)
    monkeypatch.setattr(pt, "colour", lambda ctx, dims, mu, ps, k, order: greedy_colour(dims, mu, ps, k, 0))
    monkeypatch.setattr(pt, "trace", trace)
    monkeypatch.setattr(pt, "trace_eo", trace_eo)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "evenodd", "--case", "small"])
    bench.main()
    lines = [l for l in capsys.readouterr().out.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["config"]["workload"].startswith("evenodd:") and len(d["cases"]) == 2 and d["value"] > 1.2
    for c in d["cases"]:
        assert sum(c["iters_evenodd"]) < sum(c["iters_full"]) and c["max_rel_diff"] < 1e-8, c
    assert d["trace"]["max_rel_diff"] < 1e-7 and d["trace"]["colours"] >= 2, d["trace"]


def test_multigrid_leg_json_line(monkeypatch, capsys):
    """`bench.py --workload multigrid --case small` on the CPU: plain solves
    from the oracle, multigrid ones from the library's host twins; fewer
    multigrid iterations and agreeing solutions."""
    import numpy as np
    import torch
    import types
    sys.path.insert(0, ROOT)
    import bench
    import oracle.estimator as OE
    from paper_2106_01275_gb300 import ptrace as pt

    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(pt, "Context", lambda dev: types.SimpleNamespace(device=dev, set_max_slots=lambda n: None))
    monkeypatch.setattr(pt, "laplacian", lambda ctx, dims, m2: types.SimpleNamespace(kind=0, dims=dims, m2=m2))
    monkeypatch.setattr(pt, "wilson", lambda ctx, dims, U, kappa, ap: types.SimpleNamespace(
        kind=1, dims=dims, U=np.asarray(U), kappa=kappa))

    def solve(op, b, prec, tol, maxit):
        o = OE.Laplacian(op.dims, op.m2) if op.kind == 0 else OE.Wilson(op.dims, op.U, op.kappa)
        x, it, _ = o.solve(b.numpy()[0], tol)
        return torch.as_tensor(np.asarray(x).reshape(b.shape)), np.array([it]), None, {}

    def mg_solve(op, b, block, nu, omega, tol, maxit):
        x, its, rel = pt.mg_solve_host(op.dims, op.m2, b.numpy(), block, nu, omega, tol, maxit)
        return torch.as_tensor(x), its, rel

    def wmg_solve(op, b, block, nv, sweeps, nu, omega, restart, seed, tol, maxit, csw=0.0):
        x, its, rel = pt.wmg_solve_host(op.dims, op.U, op.kappa, b.numpy(), block, nv, sweeps, nu, omega, restart,
                                        seed, tol, maxit, csw=csw)
        return torch.as_tensor(x), its, rel

    def eo_clover_blocks(op, csw):
        from oracle import evenodd as EO
        C = pt.clover_blocks_host(op.dims, op.U, op.kappa, csw)
        ev, od = EO.split(op.dims)
        return np.eye(12)[None] + C[ev], pt.site_blocks_invert_host(C[od], 1.0)

    def eo_solve(op, b, tol, maxit, blocks=None):
        x, its, rel = pt.eo_solve_host(1, op.dims, b.numpy(), tol=tol, maxit=maxit, kappa=op.kappa, U=op.U,
                                       blocks=blocks)
        return torch.as_tensor(x), its, rel

    monkeypatch.setattr(pt, "solve", solve)
    monkeypatch.setattr(pt, "mg_solve", mg_solve)
    monkeypatch.setattr(pt, "wmg_solve", wmg_solve)
    monkeypatch.setattr(pt, "eo_clover_blocks", eo_clover_blocks)
    monkeypatch.setattr(pt, "eo_solve", eo_solve)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "multigrid", "--case", "small"])
    bench.main()
    lines = [l for l in capsys.readouterr().out.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["config"]["workload"].startswith("multigrid:") and len(d["cases"]) == 3 and d["value"] > 1.0
    assert d["warmup"] == 1
    for c in d["cases"]:
        assert c["relres_multigrid"] <= 1e-10 and c["max_rel_diff"] < 1e-7, c
        assert c["seconds_multigrid_setup"] >= 0.0 and c["seconds_multigrid_solve"] >= 0.0, c
        if c["operator"] == "clover":
            assert c["iters_plain"] is None and c["iters_evenodd_bicgstab"] > 0, c
        else:
            assert c["iters_multigrid"] < c["iters_plain"], c


def test_reference_arm_clover_workload():
    """The reference arm of the clover workload times the oracle's clover
    Wilson operator (small case)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "clover24", "--case", "small", "--steps", "1", "--warmup", "3", "--cpu-seconds", "1"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"].startswith("clover24") and "c_sw=1.0" in d["config"]["workload"]
    assert "clover Wilson" in d["cpu_baseline"]["sample"]
