#!/usr/bin/env python3
"""Benchmark of the displacement-probed estimator of Tr(P A^{-1}) on one GB300.

Workload (default, "lap16"): shifted scalar Laplacian on a 16^4 lattice
(65,536 sites), m^2 = 0.01; displacements p = 0..4 along dim 3; one
displaced distance-k colouring per (p, k) for k = 1..4 (the smaller of the
natural and red-black greedy colourings, 20 colourings, 457 colours);
8 independent Z2 noise sets per colouring -> 3,656 right-hand sides per step.
One step = every probe of every colouring solved (mixed FP32 CG inside FP64
defect correction to relative residual 1e-10) and contracted with every
displacement p = 0..4, all in one batched, graph-driven engine run.

Reported value: operator applications x sites per second over the whole step
(site*RHS/s).  Also reported: the time to the standard deviation reached by
8 noise sets (= the step time), the same for the plain FP64 one-RHS-at-a-time
GPU solve on identical probes, the roofline of the dominant kernel (the FP32
stencil apply of the inner CG) against the measured HBM bandwidth, an end to
end measurement through the C ABI with host buffers, and the FP64 CPU oracle
timed on the host cores (cpu_baseline).

--impl reference times the CPU oracle itself on this workload's metric.
Multi-GPU (torchrun): every rank runs the full workload on its own noise sets
(weak scaling); there is no collective on the data path.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = [16, 16, 16, 16]
M2 = 0.01
MU = 3
P_LIST = [0, 1, 2, 3, 4]
K_LIST = [1, 2, 3, 4]
N_SETS = 8
TOL = 1e-10
MAXIT = 20000
SEED = 1000
METRIC = "time to Tr(PA^-1) at fixed sigma; stencil site*RHS/s & HBM %; mixed vs FP64 1xGB300"
# FP32 stencil apply of the inner CG, fused with the direction update
# p_i = r + beta p_{i-1}: read r and p_{i-1}, write p_i and q = A p_i (4 B each)
APPLY_BYTES_PER_SITE_RHS = 16
# DRAM bytes (read + write) per site*RHS of k_cg_apply_v4<float> from one ncu
# capture of the small case (238 RHS, all active: 125.5 MB + 85.8 MB per
# launch; profiles/k_cg_apply_v4_lap16_small.md).  Set to None whenever the
# kernel changes until it is captured again.
APPLY_NCU_TRAFFIC_PER_SITE_RHS = (125.515008e6 + 85.80608e6) / (238 * 65536)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_colourings(pt, ctx, small=False):
    """One colouring per (p, k): the smaller of natural and red-black."""
    import torch
    N = int(np.prod(DIMS))
    pk = [(0, 4)] if small else [(p, k) for k in K_LIST for p in P_LIST]
    cols = torch.empty((len(pk), N), dtype=torch.int32, device="cuda")
    m, labels = [], []
    i = 0
    for p, k in pk:
        c0, m0 = pt.colour(ctx, DIMS, MU, [p], k, "natural")
        c1, m1 = pt.colour(ctx, DIMS, MU, [p], k, "redblack")
        cols[i].copy_(c0 if m0 <= m1 else c1)
        m.append(min(m0, m1))
        labels.append((p, k))
        i += 1
    torch.cuda.synchronize()
    return cols, m, labels


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2106_01275_gb300 import ptrace as pt

    ctx = pt.Context(local)
    ctx.set_memory_budget(64 << 30)
    op = pt.laplacian(ctx, DIMS, M2)
    cols, m, labels = make_colourings(pt, ctx, args.case == "small")
    N = int(np.prod(DIMS))
    set0 = rank * N_SETS                      # weak scaling: each rank its own noise sets
    n_sets_step = 2 if args.case == "small" else N_SETS

    def step(prec="mixed_fp32", set_base=set0, n_sets=n_sets_step):
        return pt.trace_multi(op, cols, m, MU, P_LIST, "z2", SEED, set_base, n_sets, True, prec, TOL, MAXIT)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ctx.profile(True)
    ctx.profile_read(0, reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = []
    est = None
    for _ in range(args.steps):
        est, st = step()
        stats.append(st)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ctx.profile(False)
    clocks = clk.stop()
    t_ms = ev0.elapsed_time(ev1)
    apply_launches, apply_ms = ctx.profile_read(0, reset=True)
    site_rhs = sum(s["site_rhs_applies"] for s in stats)
    inner_iters = sum(s["inner_iters"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    if world > 1:
        t = torch.tensor([t_ms, float(site_rhs)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        t_ms, site_rhs_all = float(tmax[0]), float(t[1])
    else:
        site_rhs_all = float(site_rhs)
    value = site_rhs_all / (t_ms / 1e3)
    step_s = t_ms / 1e3 / args.steps

    peak, peak_kind = peaks()
    apply_bytes = inner_iters * N * APPLY_BYTES_PER_SITE_RHS
    achieved = apply_bytes / (apply_ms / 1e3) / 1e9 if apply_ms > 0 else None
    roofline = {"bound": "hbm", "kernel": "k_cg_apply<float> (FP32 p update + stencil apply + p.q dot)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": (APPLY_NCU_TRAFFIC_PER_SITE_RHS * inner_iters * N / apply_launches
                            if APPLY_NCU_TRAFFIC_PER_SITE_RHS and apply_launches else None),
                "traffic_source": "ncu dram read+write of the apply kernel on the 238-RHS case, "
                                  "scaled per site*RHS to the average launch",
                "algorithmic_bytes_per_site_rhs": APPLY_BYTES_PER_SITE_RHS,
                "launches": apply_launches, "apply_ms_total": apply_ms,
                "apply_share_of_step": apply_ms / t_ms if t_ms else None}

    out = {"metric": METRIC, "value": value, "unit": "site*RHS/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
           "config": {"workload": "lap16: 16^4 shifted Laplacian m2=0.01, p=0..4 along dim 3, "
                                  "(p,k)-colourings k=1..4 (min of natural/red-black, 457 colours), "
                                  "8 Z2 sets, mixed FP32 CG + FP64 defect correction to 1e-10",
                      "lattice": DIMS, "n_rhs_per_step": int(stats[-1]["n_rhs"]),
                      "n_colours": m, "parallelism": "rhs-batched, %d rank(s), weak" % world,
                      "l2": "working set > L2 (all RHS resident: %.1f GB)" %
                            (stats[-1]["n_slots"] * N * 24 / 1e9)},
           "gpu_launches": int(launches), "roofline": roofline, "clocks": clocks}

    if rank == 0 and world == 1 and not args.skip_baselines:
        # time to sigma: every (p, k) estimator at 8 sets reaches its sigma in one step
        sig = {}
        var = np.var(est, axis=1, ddof=1)            # [n_col, n_p]
        for i, (p, k) in enumerate(labels):
            sig["p%d_k%d" % (p, k)] = float(np.sqrt(var[i, P_LIST.index(p)] / N_SETS))
        out["time_to_sigma_s"] = step_s
        out["sigma_target"] = "sigma of the mean after 8 Z2 sets, each (p,k) estimator of Tr(P_p A^-1)"
        out["solves_per_s"] = stats[-1]["n_rhs"] / step_s
        out["mean_inner_iters_per_rhs"] = stats[-1]["inner_iters"] / stats[-1]["n_rhs"]
        # plain FP64 one-RHS-at-a-time GPU solve on identical probes: one of the 8 sets, x 8
        ctx.set_max_slots(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est64, st64 = step("fp64", set0, 1)
        torch.cuda.synchronize()
        t_plain_set = time.perf_counter() - t0
        ctx.set_max_slots(0)
        est_mixed_set0 = est[:, 0, :]
        rel = np.max(np.abs(est64[:, 0, :] - est_mixed_set0) / np.maximum(np.abs(est64[:, 0, :]), 1e-300))
        out["fp64_plain"] = {"time_to_sigma_s": t_plain_set * N_SETS, "measured_sets": 1,
                             "time_per_set_s": t_plain_set, "site_rhs_per_s": st64["site_rhs_applies"] / t_plain_set,
                             "max_rel_diff_vs_mixed": float(rel)}
        out["speedup_vs_fp64_plain"] = t_plain_set * N_SETS / step_s
        # e2e through the C ABI with host buffers: colourings copied in, estimates copied out
        cols_host = cols.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        site_e2e = 0
        for _ in range(args.steps):
            cols_dev = cols_host.to("cuda", non_blocking=True)
            est_h, st_h = pt.trace_multi(op, cols_dev, m, MU, P_LIST, "z2", SEED, set0, N_SETS, True,
                                         "mixed_fp32", TOL, MAXIT)
            site_e2e += st_h["site_rhs_applies"]
        t_e2e = time.perf_counter() - t0
        out["e2e"] = {"value": site_e2e / t_e2e, "unit": "site*RHS/s",
                      "h2d_bytes_per_step": int(cols_host.numel() * 4),
                      "d2h_bytes_per_step": int(est_h.size * 16)}
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    elif rank == 0:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_sample(seconds):
    """The oracle as it stands, on a bounded sample of the workload: probes of
    the (p, k) = (4, 1) colouring (set 0, then further sets) solved one by one
    with its FP64 CG to 1e-10 and contracted; returns site*RHS/s."""
    import oracle.estimator as OE
    from oracle.colouring import greedy_colour
    from oracle.lattice import displace
    from oracle.probes import probe
    from oracle.solvers import cg
    from oracle.operators import laplacian_apply
    col, m = greedy_colour(DIMS, MU, [4], 1, 0)
    N = int(np.prod(DIMS))
    t0 = time.perf_counter()
    site_rhs, n_rhs, s = 0, 0, 0
    while time.perf_counter() - t0 < seconds:
        for c in range(m):
            v = probe(col, c, SEED, s, 0, 1, 0)[:, 0]
            x, its, rel = cg(lambda f: laplacian_apply(f, DIMS, M2), v, TOL, MAXIT)
            _ = [np.vdot(v, displace(x, DIMS, MU, p)) for p in P_LIST]
            site_rhs += (its + 1) * N
            n_rhs += 1
            if time.perf_counter() - t0 >= seconds:
                break
        s += 1
    dt = time.perf_counter() - t0
    return site_rhs / dt, n_rhs, dt


def cpu_baseline(seconds):
    v, n_rhs, dt = oracle_sample(seconds)
    return {"value": v, "unit": "site*RHS/s", "cores": 1, "kind": "oracle",
            "sample": "%d RHS of the (p,k)=(4,1) colouring, FP64 CG to 1e-10 with contraction, %.1f s" % (n_rhs, dt)}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    per_step = max(2.0, min(20.0, args.cpu_seconds / max(args.steps, 1)))
    for _ in range(args.warmup):
        oracle_sample(min(per_step, 2.0))
    t0 = time.perf_counter()
    site, n_rhs = 0.0, 0
    for _ in range(args.steps):
        v, n, dt = oracle_sample(per_step)
        site += v * dt
        n_rhs += n
    t = time.perf_counter() - t0
    value = site / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site*RHS/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "lap16 (oracle on a bounded sample per step)", "lattice": DIMS},
           "cpu_baseline": {"value": value, "unit": "site*RHS/s", "cores": 1, "kind": "oracle",
                            "sample": "%d RHS over %d steps of %.1f s" % (n_rhs, args.steps, per_step)},
           "e2e": {"value": value, "unit": "site*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-baselines", action="store_true")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: the (p,k)=(0,4) colouring with 2 sets only (for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
