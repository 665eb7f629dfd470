#!/usr/bin/env python3
"""Benchmark of the displacement-probed estimator of Tr(P A^{-1}) on one GB300.

Default workload "lap16" (the plain-method configuration of the metric):
shifted scalar Laplacian on a 16^4 lattice (65,536 sites), m^2 = 0.01;
displacements p = 0..4 along dim 3; one displaced distance-k colouring per
(p, k), k = 1..4 (the smaller of the natural and red-black greedy colourings:
20 colourings, 457 colours); 8 independent Z2 noise sets per colouring ->
3,656 right-hand sides per step.  One step = every probe of every colouring
solved (mixed FP32 CG inside FP64 defect correction to relative residual
1e-10) and contracted with every displacement, in one batched engine run.

"wilson24": Wilson-Dirac on 24^3 x 48, kappa = 0.124, antiperiodic t, links
exp(i 0.3 H) from seed 1234; displacements p = 0, 2, 4, 8 along z with their
(p, 2) colourings, Z4 noise with 12x spin-colour dilution, 4 noise sets;
mixed FP32 BiCGStab inside FP64 defect correction to 1e-10.

"clover24": the same with the clover term, c_sw = 1.0 (the operator class of
the paper's production runs, on synthetic links), solved on the even Schur
complement S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe.

Reported value: operator applications x sites per second over the whole step
(site*RHS/s).  Also reported: the time to the standard deviation of the noise
sets of one step (= the step time), the same for the plain FP64
one-RHS-at-a-time GPU solve on identical probes, the roofline of the dominant
kernel (the stencil apply of the inner Krylov iteration, timed with CUDA
events recorded inside the solver's graph), an end-to-end measurement through
the C ABI with host buffers, and the FP64 CPU oracle on the host cores.

--impl reference times the CPU oracle itself on the workload's metric.
Multi-GPU (torchrun): every rank runs the full workload on its own noise sets
(weak scaling); no collective touches the data path.
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

from paper_2106_01275_gb300 import sharding  # noqa: E402  (imports nothing heavy)

METRIC = "time to Tr(PA^-1) at fixed sigma; stencil site*RHS/s & HBM %; mixed vs FP64 1xGB300"
TOL = 1e-10
MAXIT = 20000
SEED = 1000


class Workload:
    def __init__(self, name, kind, dims, mu, pk, p_contract, n_sets, noise, desc, m2=None, kappa=None,
                 link_seed=None, plain_subset=None, csw=0.0):
        self.name, self.kind, self.dims, self.mu, self.pk = name, kind, list(dims), mu, list(pk)
        self.csw = float(csw)                # clover coefficient (Wilson; 0: none)
        self.p_contract, self.n_sets, self.noise, self.desc = list(p_contract), n_sets, noise, desc
        self.m2, self.kappa, self.link_seed = m2, kappa, link_seed
        self.plain_subset = plain_subset     # colourings used for the plain FP64 timing (None = all)
        self.N = int(np.prod(dims))

    # algorithmic bytes of the inner apply (FP32), per site*RHS and per site*launch
    def apply_bytes(self, evenodd=False):
        if self.kind == "lap":
            # full system: read r, p_{i-1}; write p_i, q.  Even-odd, per lattice site: the odd-site
            # hop reads r, p_{i-1} at the even sites and writes t (6 B), the even-site apply reads
            # r, p_{i-1}, t and writes p_i, q (10 B)
            return 16.0, 0.0
        if not evenodd:
            # per apply, averaged over the two of a BiCGStab iteration: v = A p also reads
            # r0 for (r0, v) -> 3 x 96 B; t = A s -> 2 x 96 B; plus the 4 x 2 x 9 FP32
            # complex links once per launch
            return 240.0, 288.0
        # even-odd, per lattice site: the odd-site hop reads p (or s) at the even sites and
        # writes h at the odd ones (96 B); v = S p then reads h, p, r0 and writes v (192 B),
        # t = S s reads h, s and writes t (144 B); every link is read by both kernels; with the
        # clover term the hop also reads A_oo^{-1} (288 B per odd site) and the apply A_ee
        # (288 B per even site)
        return 264.0, 576.0 + (288.0 if self.csw else 0.0)


def workloads(case):
    small = case == "small"
    lap = Workload(
        "lap16", "lap", [16, 16, 16, 16], 3,
        [(0, 4)] if small else [(p, k) for k in (1, 2, 3, 4) for p in (0, 1, 2, 3, 4)],
        [0, 1, 2, 3, 4], 2 if small else 8, "z2",
        "lap16: 16^4 shifted Laplacian m2=0.01, p=0..4 along dim 3, (p,k)-colourings k=1..4 "
        "(min of natural/red-black, 457 colours), 8 Z2 sets, mixed FP32 CG + FP64 defect correction to 1e-10"
        if not small else "lap16 small: (p,k)=(0,4) colouring, 2 Z2 sets", m2=0.01)
    wil = Workload(
        "wilson24", "wil", [16, 16, 16, 32] if small else [24, 24, 24, 48], 2,
        [(4, 2)] if small else [(0, 2), (2, 2), (4, 2), (8, 2)], [0, 2, 4, 8], 1 if small else 4, "z4",
        "wilson24: Wilson-Dirac 24^3x48 kappa=0.124 antiperiodic t, p=0,2,4,8 along z with (p,2)-colourings, "
        "Z4 x 12 spin-colour dilution, 4 sets (1584 RHS), mixed FP32 BiCGStab + FP64 defect correction to 1e-10"
        if not small else "wilson24 small: 16^3x32, (p,k)=(4,2), 1 Z4 set, 12x dilution",
        kappa=0.124, link_seed=1234, plain_subset=[3])
    clv = Workload(
        "clover24", "wil", wil.dims, 2, wil.pk, wil.p_contract, wil.n_sets, "z4",
        ("clover24: clover Wilson-Dirac c_sw=1.0 24^3x48 kappa=0.124 antiperiodic t, p=0,2,4,8 along z with "
         "(p,2)-colourings, Z4 x 12 spin-colour dilution, 4 sets (1584 RHS), mixed FP32 BiCGStab on the even "
         "Schur complement + FP64 defect correction to 1e-10")
        if not small else "clover24 small: 16^3x32 c_sw=1.0, (p,k)=(4,2), 1 Z4 set, 12x dilution",
        kappa=0.124, link_seed=1234, plain_subset=[3], csw=1.0)
    return {"lap16": lap, "wilson24": wil, "clover24": clv}


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


def make_colourings(pt, ctx, W):
    """One colouring per (p, k): the smaller of natural and red-black."""
    import torch
    cols = torch.empty((len(W.pk), W.N), dtype=torch.int32, device="cuda")
    m = []
    for i, (p, k) in enumerate(W.pk):
        c0, m0 = pt.colour(ctx, W.dims, W.mu, [p], k, "natural")
        c1, m1 = pt.colour(ctx, W.dims, W.mu, [p], k, "redblack")
        cols[i].copy_(c0 if m0 <= m1 else c1)
        m.append(min(m0, m1))
    torch.cuda.synchronize()
    return cols, m


def make_operator(pt, ctx, W):
    import torch
    if W.kind == "lap":
        return pt.laplacian(ctx, W.dims, W.m2)
    from paper_2106_01275_gb300 import inputs
    U = torch.as_tensor(inputs.gauge_links(W.dims, W.link_seed)).cuda()
    op = pt.wilson(ctx, W.dims, U, W.kappa, True)
    if W.csw:
        pt.set_clover(op, W.csw)
    return op


def dist_backend():
    """NCCL between GPUs; gloo where no GPU is visible (CPU runs of the same
    multi-rank path, with the binding stood in for)."""
    import torch
    return "nccl" if torch.cuda.is_available() else "gloo"


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    backend = dist_backend()
    red_dev = "cuda" if backend == "nccl" else "cpu"
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend)
    torch.cuda.set_device(local)
    from paper_2106_01275_gb300 import ptrace as pt

    W = workloads(args.case)[args.workload]
    ctx = pt.Context(local)
    ctx.set_memory_budget((200 if W.kind == "wil" else 64) << 30)
    op = make_operator(pt, ctx, W)
    cols, m = make_colourings(pt, ctx, W)
    N = W.N
    set0, _ = sharding.rank_sets(rank, W.n_sets)      # weak scaling: each rank its own noise sets

    def step(prec=args.prec, set_base=set0, n_sets=W.n_sets, c=cols, mm=m):
        return pt.trace_multi(op, c, mm, W.mu, W.p_contract, W.noise, SEED, set_base, n_sets, True, prec,
                              TOL, MAXIT)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # autotune the engine on trial probes of the largest colouring (set-up, untimed)
    big = int(np.argmax(m))
    tuning = pt.autotune(op, cols[big].contiguous(), m[big], W.mu, W.noise, SEED + 7, args.prec, TOL, MAXIT,
                         64 if W.kind == "lap" else 24) if not args.no_tune else pt.get_tuning(op, args.prec)
    if args.tuning:                  # explicit engine parameters on top of the tuned ones
        fixed = {k: (float(v) if k == "delta" else int(v))
                 for k, v in (kv.split("=") for kv in args.tuning.split(","))}
        pt.set_tuning(op, args.prec, **fixed)
        tuning = pt.get_tuning(op, args.prec)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ctx.profile(True)
    for c in range(4):
        ctx.profile_read(c, reset=True)
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
    prof = [ctx.profile_read(c, reset=True) for c in range(4)]
    apply_launches, apply_ms = prof[0]
    site_rhs = sum(s["site_rhs_applies"] for s in stats)
    inner_iters = sum(s["inner_iters"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    t_ms, site_rhs_all = sharding.reduce_timing(t_ms, site_rhs, red_dev)
    value = site_rhs_all / (t_ms / 1e3)
    step_s = t_ms / 1e3 / args.steps

    peak, peak_kind = peaks()
    eo = bool(tuning.get("evenodd", 0)) and all(d % 2 == 0 for d in W.dims)
    b_rhs, b_launch = W.apply_bytes(eo)
    if args.prec == "mixed_bf16":              # half the bytes of every inner vector and link
        b_rhs, b_launch = b_rhs / 2, (b_launch / 2 if W.kind == "lap" else 36 * 4.0 * (2 if eo else 1))
    applies_per_iter = 1 if W.kind == "lap" else 2
    apply_bytes = inner_iters * applies_per_iter * N * b_rhs + apply_launches * N * b_launch
    achieved = apply_bytes / (apply_ms / 1e3) / 1e9 if apply_ms > 0 else None
    if W.kind == "lap":
        kernel = ("k_eo_hop_v4 + k_eo_apply_v4 <float> (S p = d p - H_eo H_oe p / d on the even sites, p update, "
                  "p.q)" if eo else "k_cg_apply_v4<float> (p update + stencil + p.q)")
    elif eo and W.csw:
        kernel = ("k_weo_hop + k_weo_apply1/2 <float,float,clover> (S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe on the "
                  "even sites + BiCGStab dots)")
    elif eo and tuning.get("rhs_block", 1) == 8 and tuning.get("cta_threads", 0) in (0, 256):
        kernel = ("k_weo_hop_g + k_weo_apply1/2_g <float,float> (eight slots per item, links staged in shared "
                  "memory; S = 1 - kappa^2 D_eo D_oe on the even sites + BiCGStab dots)")
    elif eo:
        kernel = ("k_weo_hop + k_weo_apply1/2 <float,float> (S = 1 - kappa^2 D_eo D_oe on the even sites + "
                  "BiCGStab dots)")
    elif tuning.get("rhs_block", 1) == 2:
        kernel = "k_bicg_apply1/2_x2<float,float> (Wilson apply for two right-hand sides per item + dots)"
    else:
        kernel = "k_bicg_apply1/2<float,float> (Wilson apply + dots)"
    roofline = {"bound": "hbm", "kernel": kernel,
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": None,
                "traffic_source": "not sampled in this run: the ncu DRAM bytes of the apply are in the profile "
                                  "summaries committed beside the kernels",
                "algorithmic_bytes_per_site_rhs": b_rhs, "algorithmic_bytes_per_site_launch": b_launch,
                "launches": apply_launches, "apply_ms_total": apply_ms,
                "apply_share_of_step": apply_ms / t_ms if t_ms else None,
                "step_breakdown_ms": {"apply": prof[0][1], "inner_vector": prof[1][1], "outer_fp64": prof[2][1],
                                      "all_iterations": prof[3][1]}}
    if eo and W.kind == "lap":
        roofline["bytes_note"] = ("per inner iteration and lattice site: k_eo_hop reads r, p_{i-1} at the even "
                                  "sites and writes t at the odd ones (6 B), k_eo_apply reads r, p_{i-1}, t and "
                                  "writes p_i, q (10 B)")
    elif eo:
        roofline["bytes_note"] = ("per S application and lattice site: k_weo_hop 96 B, k_weo_apply1 192 B / "
                                  "k_weo_apply2 144 B (averaged: 264 B), links 2 x 288 B per site per application"
                                  + (", clover blocks 288 B per site per application (A_oo^{-1} on the odd "
                                     "sites, A_ee on the even ones)" if W.csw else ""))
    if W.kind == "lap":
        n_vec, vec_sites = (6, N // 2) if eo else (5, N)
    else:
        n_vec, vec_sites = (8, N // 2) if eo else (7, N)

    out = {"metric": METRIC, "value": value, "unit": "site*RHS/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 inner / f64 outer" if args.prec == "mixed_fp32" else "bf16 storage, f32 arith / f64 outer",
           "data": "synthetic",
           "config": {"workload": W.desc, "lattice": W.dims, "n_rhs_per_step": int(stats[-1]["n_rhs"]),
                      "n_colours": m, "parallelism": "rhs-batched, %d rank(s), weak" % world,
                      "tuning": tuning,
                      "solver": ("even-odd (Schur complement on the even sites)" if eo else "full system"),
                      "l2": "working set > L2 (resident RHS: %d, %.1f GB of inner vectors)" %
                            (stats[-1]["n_slots"], stats[-1]["n_slots"] * vec_sites * n_vec *
                             (4 if W.kind == "lap" else 96) / 1e9)},
           "gpu_launches": int(launches), "roofline": roofline, "clocks": clocks,
           "mean_inner_iters_per_rhs": stats[-1]["inner_iters"] / stats[-1]["n_rhs"],
           "mean_outer_iters_per_rhs": stats[-1]["outer_iters"] / stats[-1]["n_rhs"],
           "solves_per_s": stats[-1]["n_rhs"] / step_s,
           "max_true_relres": stats[-1]["max_relres"]}
    if est is not None and W.n_sets > 1:
        # the standard deviation of the mean over the step's noise sets for every (p, k) estimator and
        # displacement: the sigma that one step reaches (the plain FP64 arm solves the same probes)
        e = np.asarray(est)
        var_s = (np.abs(e - e.mean(axis=1, keepdims=True)) ** 2).sum(axis=1) / (e.shape[1] - 1)
        sig = np.sqrt(var_s / e.shape[1])
        out["sigma_mean"] = {"rows": ["(%d,%d)" % tuple(pk) for pk in W.pk],
                             "cols": ["p=%d" % q for q in W.p_contract],
                             "values": [[float("%.6g" % v) for v in row] for row in sig],
                             "relative": [[float("%.4g" % v) for v in row]
                                          for row in sig / np.maximum(np.abs(e.mean(axis=1)), 1e-300)],
                             "n_sets": int(e.shape[1])}
        # Eq. (17): sqrt(v m / M) / |Tr(P_n A^-1)| for every colouring and displacement, v the sample
        # variance of the colouring's estimator over the step's noise sets, M the largest colour count,
        # the trace taken as the mean over every colouring and set
        e = np.asarray(est)                                            # [n_col, n_sets, n_p]
        var = (np.abs(e - e.mean(axis=1, keepdims=True)) ** 2).sum(axis=1) / (e.shape[1] - 1)
        tr = np.abs(e.mean(axis=(0, 1)))
        M = max(m)
        nre = np.sqrt(var * np.asarray(m, dtype=float)[:, None] / M) / np.maximum(tr[None, :], 1e-300)
        best = {("p=%d" % W.p_contract[n]): "(%d,%d)" % tuple(W.pk[int(np.argmin(nre[:, n]))])
                for n in range(len(W.p_contract))}
        out["normalised_relative_error"] = {
            "rows": ["(%d,%d)" % tuple(pk) for pk in W.pk], "cols": ["p=%d" % q for q in W.p_contract],
            "values": np.round(nre, 8).tolist(), "best_colouring_per_displacement": best}

    if W.kind == "lap" and rank == 0:
        # the hierarchical reading of "k = 1..4 grown at runtime": colourings nested level by level
        # (pt_colour_nested), reported beside the independent ones the step solves
        nested, levels = {}, []
        for p in sorted({pk[0] for pk in W.pk}):
            ks = sorted(k for (pp, k) in W.pk if pp == p)
            if ks != list(range(1, ks[-1] + 1)):
                continue
            par, mp_ = pt.colour(ctx, W.dims, W.mu, [p], 1, "natural")
            lev, counts = [par.clone()], [mp_]
            for k in ks[1:]:
                par, mp_ = pt.colour_nested(ctx, W.dims, W.mu, [p], k, par, mp_, "natural")
                lev.append(par.clone())
                counts.append(mp_)
            nested["p=%d" % p] = counts
            levels.append((torch.stack(lev).contiguous(), counts))
        if nested:
            out["config"]["nested_colours_natural_k1_up"] = nested
            # every level's estimate from the finest level's solves only (pt_trace_PAinv_nested),
            # same noise sets and displacements as the step
            def nested_run(s0):
                n_rhs = 0
                for cols_l, counts in levels:
                    _, stn = pt.trace_nested(op, cols_l, counts, W.mu, W.p_contract, W.noise, SEED, s0, W.n_sets,
                                             True, args.prec, TOL, MAXIT)
                    n_rhs += stn["n_rhs"]
                return n_rhs
            nested_run(set0)                                   # warm-up (work space, graphs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n_rhs_nested = nested_run(set0)
            torch.cuda.synchronize()
            t_nested = time.perf_counter() - t0
            out["nested"] = {"time_s": t_nested, "n_rhs": int(n_rhs_nested),
                             "estimates": "k = 1..%d for every p, %d sets, from the finest level's solves"
                                          % (len(levels[0][1]), W.n_sets),
                             "independent_step_s": step_s, "independent_n_rhs": int(stats[-1]["n_rhs"])}

    if rank == 0 and world == 1 and not args.skip_baselines:
        # time to sigma: the estimators reach the sigma of their W.n_sets sets in one step
        out["time_to_sigma_s"] = step_s
        out["sigma_target"] = ("sigma_mean above: the standard deviation of the mean over the %d noise sets of "
                               "one step, for every (p,k) estimator and displacement; the plain arm solves the "
                               "same probes and reaches the same values" % W.n_sets)
        # plain FP64 one-RHS-at-a-time GPU solve on identical probes, on the full system (no even-odd):
        # every colouring and set for the Laplacian; for Wilson one colouring and one set, scaled
        sub = W.plain_subset if W.plain_subset is not None else list(range(len(m)))
        csub = cols[sub].contiguous()
        msub = [m[i] for i in sub]
        n_sets_plain = W.n_sets if W.kind == "lap" else 1
        ctx.set_max_slots(1)
        pt.set_tuning(op, "fp64", evenodd=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est64, st64 = step("fp64", set0, n_sets_plain, csub, msub)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        ctx.set_max_slots(0)
        pt.set_tuning(op, "fp64", reset=True)
        frac = st64["n_rhs"] / stats[-1]["n_rhs"]          # share of the step's right-hand sides timed
        t_plain_step = t_plain / frac
        ref = est[sub][:, :n_sets_plain, :]
        rel = np.max(np.abs(est64 - ref) / np.maximum(np.abs(est64), 1e-300))
        out["fp64_plain"] = {"time_to_sigma_s": t_plain_step, "measured_rhs": int(st64["n_rhs"]),
                             "measured_s": t_plain, "scaled_by_rhs_fraction": frac,
                             "solver": ("FP64 BiCGStab on the even Schur complement (the clover operator has no "
                                        "full-system path), one right-hand side at a time" if W.csw else
                                        "FP64 CG / BiCGStab on the full system, one right-hand side at a time"),
                             "site_rhs_per_s": st64["site_rhs_applies"] / t_plain,
                             "max_rel_diff_vs_mixed": float(rel)}
        out["speedup_vs_fp64_plain"] = t_plain_step / step_s
        # e2e through the C ABI with host buffers: colourings copied in, estimates copied out
        cols_host = cols.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        site_e2e = 0
        for _ in range(args.steps):
            cols_dev = cols_host.to("cuda", non_blocking=True)
            est_h, st_h = step(c=cols_dev)
            site_e2e += st_h["site_rhs_applies"]
        t_e2e = time.perf_counter() - t0
        out["e2e"] = {"value": site_e2e / t_e2e, "unit": "site*RHS/s",
                      "h2d_bytes_per_step": int(cols_host.numel() * 4),
                      "d2h_bytes_per_step": int(est_h.size * 16)}
        out["cpu_baseline"] = cpu_baseline(W, args.cpu_seconds)
    elif rank == 0:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_grad(args):
    """Adjoint-gradient workload: Wilson-Dirac 32^3 x 64 (small: 16^3 x 32),
    kappa = 0.12, p = 4 along z with its (4, 2) colouring, one Z4 set with 12x
    dilution; per step every probe is solved forward and adjoint (mixed FP32
    BiCGStab + FP64 defect correction to 1e-10), no Krylov history is kept,
    and dT/dkappa and the per-link derivatives G, Gbar are formed."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        torch.distributed.init_process_group(dist_backend())
    torch.cuda.set_device(local)
    from paper_2106_01275_gb300 import inputs
    from paper_2106_01275_gb300 import ptrace as pt
    dims = [16, 16, 16, 32] if args.case == "small" else [32, 32, 32, 64]
    kappa, mu, p, k = 0.12, 2, 4, 2
    N = int(np.prod(dims))
    ctx = pt.Context(local)
    ctx.set_memory_budget(200 << 30)
    U = torch.as_tensor(inputs.gauge_links(dims, 4321)).cuda()
    op = pt.wilson(ctx, dims, U, kappa, True)
    c0, m0 = pt.colour(ctx, dims, mu, [p], k, "natural")
    c1, m1 = pt.colour(ctx, dims, mu, [p], k, "redblack")
    col, m = (c0, m0) if m0 <= m1 else (c1, m1)
    set0, _ = sharding.rank_sets(rank, 1)

    def step(c=col):
        return pt.grad(op, c, m, mu, p, "z4", SEED, set0, 1, True, "mixed_fp32", TOL, MAXIT, links=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    ctx.profile(True)
    for c in range(4):
        ctx.profile_read(c, reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = []
    for _ in range(args.steps):
        est, dk, G, Gb, st = step()
        stats.append(st)
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctx.profile(False)
    clocks = clk.stop()
    t_ms = ev0.elapsed_time(ev1)
    prof = [ctx.profile_read(c, reset=True) for c in range(4)]
    site_rhs = sum(s["site_rhs_applies"] for s in stats)
    inner = sum(s["inner_iters"] for s in stats)
    t_ms, site_rhs = sharding.reduce_timing(t_ms, site_rhs, "cuda" if dist_backend() == "nccl" else "cpu")
    peak, peak_kind = peaks()
    apply_bytes = inner * 2 * N * 240.0 + prof[0][0] * N * 288.0
    achieved = apply_bytes / (prof[0][1] / 1e3) / 1e9 if prof[0][1] > 0 else None
    out = {"metric": METRIC, "value": site_rhs / (t_ms / 1e3), "unit": "site*RHS/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
           "config": {"workload": "grad32: adjoint gradient of the probed Tr(P_4 A^-1), Wilson-Dirac %s kappa=0.12, "
                                  "(4,2)-colouring (%d colours), 1 Z4 set x 12 dilution, forward + adjoint solves, "
                                  "dT/dkappa and per-link G, Gbar" % ("x".join(map(str, dims)), m),
                      "lattice": dims, "n_rhs_per_step": int(stats[-1]["n_rhs"]), "n_colours": m,
                      "parallelism": "rhs-batched, %d rank(s), weak" % world},
           "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
           "roofline": {"bound": "hbm", "kernel": "k_bicg_apply1/2<float,float>", "achieved": achieved,
                        "peak": peak, "unit": "GB/s", "frac": achieved / peak if achieved else None,
                        "peak_source": peak_kind, "traffic": None,
                        "algorithmic_bytes_per_site_rhs": 240.0, "algorithmic_bytes_per_site_launch": 288.0,
                        "step_breakdown_ms": {"apply": prof[0][1], "inner_vector": prof[1][1],
                                              "outer_fp64": prof[2][1], "all_iterations": prof[3][1]}},
           "clocks": clocks, "dT_dkappa": [dk.real, dk.imag], "estimate": [float(est.sum().real), float(est.sum().imag)],
           "mean_inner_iters_per_rhs": stats[-1]["inner_iters"] / stats[-1]["n_rhs"],
           "solves_per_s": stats[-1]["n_rhs"] / (t_ms / 1e3 / args.steps)}
    if rank == 0 and world == 1 and not args.skip_baselines:
        cols_host = col.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        site_e2e = 0
        for _ in range(args.steps):
            est_h, dk_h, G_h, Gb_h, st_h = step(cols_host.to("cuda", non_blocking=True))
            G_host, Gb_host = G_h.cpu(), Gb_h.cpu()
            site_e2e += st_h["site_rhs_applies"]
        t_e2e = time.perf_counter() - t0
        out["e2e"] = {"value": site_e2e / t_e2e, "unit": "site*RHS/s", "h2d_bytes_per_step": int(N * 4),
                      "d2h_bytes_per_step": int(G_host.numel() * 16 * 2 + 16 * 2)}
        W = Workload("grad32", "wil", dims, mu, [(p, k)], [p], 1, "z4", "", kappa=kappa, link_seed=4321)
        out["cpu_baseline"] = cpu_baseline(W, args.cpu_seconds)
        out["fp64_plain"] = None
    elif rank == 0:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def run_colour(args):
    """Displaced greedy colouring of every Table 2 tile (Sec. 3.5) on the GPU,
    natural and red-black orders, against the paper's colour counts (Table 4)
    and its single-thread seconds (Table 3).  Tiles are printed as (z, x, y, t)
    with the displacement along z; here the lattice is (x, y, z, t), mu = 2."""
    import torch
    from paper_2106_01275_gb300 import ptrace as pt
    world, rank, local = dist_setup()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ctx = pt.Context(local)
    tiles = {}
    for r in _golden("table4_colours.txt"):
        p, k, tz, tx, ty, tt, colours, lb = map(int, r)
        tiles[(p, k)] = ([tx, ty, tz, tt], colours)
    for r in _golden("table4_colours_k8_10.txt"):
        tiles[(int(r[0]), int(r[1]))] = ([32, 32, 32, 32], int(r[2]))
    t3 = {}
    for r in _golden("table3_times.txt"):
        for p in range(9):
            t3[(p, int(r[0]))] = float(r[1 + p])
    kmax = 10 if args.case == "full" else 7
    rows, t_gpu, t_cpu, match = [], 0.0, 0.0, 0
    for k in range(1, kmax + 1):
        for p in range(9):
            dims, want = tiles[(p, k)]
            t0 = time.perf_counter()
            _, m0 = pt.colour(ctx, dims, 2, [p], k, "natural")
            t1 = time.perf_counter()
            _, m1 = pt.colour(ctx, dims, 2, [p], k, "redblack")
            t2 = time.perf_counter()
            m = min(m0, m1)
            tg = (t1 - t0) if m0 <= m1 else (t2 - t1)      # time of the colouring that is kept
            rows.append({"p": p, "k": k, "tile": dims, "colours": m, "paper": want, "natural": m0,
                         "redblack": m1, "gpu_s": round(tg, 4), "paper_cpu_s": t3[(p, k)]})
            t_gpu += tg
            t_cpu += t3[(p, k)]
            match += int(m == want)
    out = {"metric": "displaced greedy colouring of the Table 2 tiles: colours vs Table 4, seconds vs Table 3",
           "value": t_cpu / t_gpu, "unit": "x (paper single-thread seconds / GB300 seconds, summed)",
           "higher_is_better": True, "n_gpus": 1, "steps": 1, "warmup": 0, "data": "synthetic",
           "config": {"workload": "Table 2 tiles, k = 1..%d, p = 0..8, displacement along z" % kmax},
           "gpu_seconds_total": t_gpu, "paper_cpu_seconds_total": t_cpu,
           "colour_counts_matching_table4": "%d of %d" % (match, len(rows)), "per_tile": rows}
    print(json.dumps(out), flush=True)


def run_deflation(args):
    """Deflation of the lowest modes (Sec. 2.4, Eq. (6)) on an 8^4 shifted
    Laplacian (m2 = 0.01 as lap16, p = 0..4 along dim 3): the device
    singular-triplet solver (block Lanczos, 33 modes = the 1 + 8 + 24 lowest
    plane waves, block 32, 24 steps), the engine's probed estimates on the
    distance-1 colouring of the union of the five displacements, and the
    deflation terms.  Reports, per displacement, the
    variance over noise sets of the plain probed estimate and of the deflated
    one (Tr(M U^H P V) + est - corr), the seconds of each part, and two checks
    at full size: the Ritz values against the closed-form plane-wave spectrum
    and Tr(M U^H V) = sum 1 / s at p = 0."""
    import itertools
    import torch
    from paper_2106_01275_gb300 import ptrace as pt
    world, rank, local = dist_setup()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ctx = pt.Context(local)
    L = 8
    dims, m2, mu, ps, k = [L] * 4, 0.01, 3, [0, 1, 2, 3, 4], 1
    n_ev, block, n_iter, n_sets = 33, 32, 24, 4 if args.case == "small" else 16
    N = L ** 4
    op = pt.laplacian(ctx, dims, m2)
    col, m = pt.colour(ctx, dims, mu, ps, k, "natural")
    start = torch.as_tensor(np.random.default_rng(SEED).standard_normal((block, N, 1)).astype(np.complex128)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U, s, V = pt.singular_triplets(op, n_ev, block, n_iter, start)
    t_eig = time.perf_counter() - t0
    want = np.array(sorted(m2 + sum(4 * np.sin(np.pi * q / L) ** 2 for q in qs)
                           for qs in itertools.product(range(L), repeat=4))[:n_ev])
    M = np.diag(1.0 / s)
    t0 = time.perf_counter()
    est, _, _, st = pt.trace(op, col, m, mu, ps, "z2", SEED, 0, n_sets, True, "mixed_fp32", 1e-10, 20000)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    corr, exact = pt.deflation_terms(op, col, m, mu, ps, "z2", SEED, 0, n_sets, U, V, M)
    t_defl = time.perf_counter() - t0
    defl = exact[None, :] + est - corr
    var_plain = est.real.var(axis=0, ddof=1)
    var_defl = defl.real.var(axis=0, ddof=1)
    out = {"metric": "deflation of the 33 lowest modes: variance of the probed Tr(P A^-1) over noise sets, "
                     "plain / deflated, per displacement",
           "value": float(np.mean(var_plain / var_defl)), "unit": "x (variance ratio, mean over p = 0..4)",
           "higher_is_better": True, "n_gpus": 1, "steps": 1, "warmup": 0, "data": "synthetic",
           "config": {"workload": "deflation: %d^4 shifted Laplacian m2=0.01, p=0..4 along dim 3, distance-1 "
                                  "colouring of their union (%d colours), %d Z2 sets, 33 modes from block "
                                  "Lanczos (block 32, 24 steps)" % (L, m, n_sets)},
           "var_plain": var_plain.tolist(), "var_deflated": var_defl.tolist(),
           "mean_plain": est.real.mean(axis=0).tolist(), "mean_deflated": defl.real.mean(axis=0).tolist(),
           "deflated_part": exact.real.tolist(),
           "seconds": {"triplets": t_eig, "solves": t_solve, "deflation_terms": t_defl},
           "n_rhs": int(st["n_rhs"]) if "n_rhs" in st else None,
           "check_ritz_vs_closed_form_max_rel": float(np.max(np.abs(s / want - 1))),
           "check_p0_trace_minus_sum_inv_s": float(abs(exact[0] - np.sum(1.0 / s)))}
    print(json.dumps(out), flush=True)


def _timed(fn, warm=1):
    """(result, seconds) of fn() after `warm` untimed calls, with a device
    synchronisation on both sides of the timed call."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def run_evenodd(args):
    """Even-odd preconditioning against the full system, both in FP64 one
    right-hand side at a time: the engine's plain solve (pt_solve, FP64, one
    slot) and the even-odd building-block solver (pt_eo_solve) on the same
    seeded right-hand sides, for the lap16 lattice (16^4 Laplacian,
    m2 = 0.01, CG) and a 16^3 x 32 Wilson lattice (kappa = 0.124, BiCGStab).
    Reports iterations, seconds (each arm warmed up once) and the largest
    difference of the solutions (relative to their largest entry)."""
    import torch
    from paper_2106_01275_gb300 import inputs
    from paper_2106_01275_gb300 import ptrace as pt
    world, rank, local = dist_setup()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ctx = pt.Context(local)
    small = args.case == "small"
    rng = np.random.default_rng(SEED)
    rows = []
    cases = [("laplacian", [8, 8, 8, 8] if small else [16, 16, 16, 16], 0.01, None),
             ("wilson", [8, 8, 8, 8] if small else [16, 16, 16, 32], None, 0.124)]
    for kind, dims, m2, kappa in cases:
        N = int(np.prod(dims))
        if kind == "laplacian":
            op = pt.laplacian(ctx, dims, m2)
            b = torch.as_tensor(rng.standard_normal((2, N))).cuda()
        else:
            op = pt.wilson(ctx, dims, torch.as_tensor(inputs.gauge_links(dims, 1234)).cuda(), kappa, True)
            b = torch.as_tensor(rng.standard_normal((2, N, 4, 3)) + 1j * rng.standard_normal((2, N, 4, 3))).cuda()
        ctx.set_max_slots(1)
        (xf, itf, _, _), t_full = _timed(lambda: pt.solve(op, b, "fp64", 1e-10, 100000))
        ctx.set_max_slots(0)
        (xe, ite, rele), t_eo = _timed(lambda: pt.eo_solve(op, b, 1e-10, 100000))
        diff = float((xf - xe).abs().max() / xe.abs().max())
        rows.append({"operator": kind, "lattice": dims, "iters_full": [int(v) for v in itf],
                     "iters_evenodd": [int(v) for v in ite], "seconds_full": t_full, "seconds_evenodd": t_eo,
                     "even_relres": [float(v) for v in rele], "max_rel_diff": diff})
    # the Laplacian trace on the same probes: the engine on the full system
    # against the even-odd trace (mixed precision both, tolerance 1e-10)
    dims = [8, 8, 8, 8] if small else [16, 16, 16, 16]
    op = pt.laplacian(ctx, dims, 0.01)
    col, m = pt.colour(ctx, dims, 3, [4], 2, "natural")
    ps = [0, 1, 2, 3, 4]
    (est_f, _, _, st_f), t_f = _timed(lambda: pt.trace(op, col, m, 3, ps, "z2", SEED, 0, 8, True, "mixed_fp32",
                                                       1e-10, 20000))
    (est_e, st_e), t_e = _timed(lambda: pt.trace_eo(op, col, m, 3, ps, "z2", SEED, 0, 8, 1e-10, 20000, 1e-5))
    trace_row = {"lattice": dims, "colours": int(m), "sets": 8, "seconds_engine_full": t_f,
                 "seconds_evenodd": t_e, "inner_iters_full": int(st_f["inner_iters"]),
                 "inner_iters_evenodd": int(st_e["inner_iters"]),
                 "max_rel_diff": float(np.abs(est_e - est_f).max() / np.abs(est_f).max())}
    out = {"metric": "even-odd preconditioning: Krylov iterations and seconds of FP64 solves, full system vs even "
                     "Schur complement", "value": float(np.mean([sum(r["iters_full"]) / sum(r["iters_evenodd"])
                                                                   for r in rows])),
           "unit": "x (iterations full / even-odd, mean over operators)", "higher_is_better": True, "n_gpus": 1,
           "steps": 1, "warmup": 1, "data": "synthetic",
           "config": {"workload": "evenodd: %s, 2 Gaussian right-hand sides each, FP64 to 1e-10, one right-hand "
                                  "side at a time" % "; ".join("%s %s" % (r["operator"], "x".join(map(str, r["lattice"])))
                                                               for r in rows)},
           "cases": rows, "trace": trace_row}
    print(json.dumps(out), flush=True)


def run_multigrid(args):
    """Two-level multigrid against the engine's plain FP64 solves (one slot),
    same seeded right-hand sides: the Laplacian at m2 = 0.001 on 16^4 (CG
    against multigrid-preconditioned CG) and Wilson at kappa = 0.124 on
    16^3 x 32 with and without the clover term (BiCGStab against adaptive
    multigrid FGMRES).  Every arm runs once untimed first.  The multigrid
    time is split into the set-up (near-null vectors, prolongator, coarse
    stencil: a call with a zero right-hand side, which returns right after
    the set-up) and the solve (the rest).  The engine has no clover
    operator, so the clover row has no plain arm; the even-odd BiCGStab on
    the clover Schur complement (pt_eo_solve) is timed beside it instead and
    the row is left out of the mean.  Reports iterations, seconds and the
    largest difference of the solutions (relative to their largest entry)."""
    import torch
    from paper_2106_01275_gb300 import inputs
    from paper_2106_01275_gb300 import ptrace as pt
    world, rank, local = dist_setup()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ctx = pt.Context(local)
    small = args.case == "small"
    rng = np.random.default_rng(SEED)
    rows = []
    dl = [8, 8, 8, 8] if small else [16, 16, 16, 16]
    dw = [4, 4, 4, 4] if small else [16, 16, 16, 32]
    cases = [("laplacian", dl, 0.001, 0.0), ("wilson", dw, 0.124, 0.0), ("clover", dw, 0.124, 1.0)]
    for kind, dims, par, csw in cases:
        N = int(np.prod(dims))
        if kind == "laplacian":
            op = pt.laplacian(ctx, dims, par)
            b = torch.as_tensor(rng.standard_normal((1, N))).cuda()
        else:
            op = pt.wilson(ctx, dims, torch.as_tensor(inputs.gauge_links(dims, 1234)).cuda(), par, True)
            b = torch.as_tensor(rng.standard_normal((1, N, 4, 3)) + 0j).cuda()
        row = {"operator": kind, "lattice": dims, "iters_plain": None, "seconds_plain": None, "max_rel_diff": None}
        if csw == 0.0:
            ctx.set_max_slots(1)
            (xf, itf, _, _), t_full = _timed(lambda: pt.solve(op, b, "fp64", 1e-10, 100000))
            ctx.set_max_slots(0)
            row.update(iters_plain=int(itf[0]), seconds_plain=t_full)
        else:
            blocks = pt.eo_clover_blocks(op, csw)
            (xf, itf, _), t_eo = _timed(lambda: pt.eo_solve(op, b, 1e-10, 100000, blocks))
            row.update(plain="none (the engine has no clover operator)", iters_evenodd_bicgstab=int(itf[0]),
                       seconds_evenodd_bicgstab=t_eo)
        if kind == "laplacian":
            (xm, itm, relm), t_mg = _timed(lambda: pt.mg_solve(op, b, 2, 2, 0.8, 1e-10, 10000))
            t_setup = 0.0                  # closed-form coarse operator: no set-up
        else:
            mg = lambda rhs: pt.wmg_solve(op, rhs, 2, 4, 20, 2, 0.8, 30, SEED, 1e-10, 5000, csw=csw)
            (xm, itm, relm), t_mg = _timed(lambda: mg(b))
            _, t_setup = _timed(lambda: mg(torch.zeros_like(b)), warm=0)
        row.update(iters_multigrid=int(itm[0]), seconds_multigrid=t_mg, seconds_multigrid_setup=t_setup,
                   seconds_multigrid_solve=max(t_mg - t_setup, 0.0), relres_multigrid=float(relm[0]),
                   max_rel_diff=float((xf - xm).abs().max() / xm.abs().max()))
        rows.append(row)
    ratios = [r["iters_plain"] / r["iters_multigrid"] for r in rows if r["iters_plain"]]
    out = {"metric": "two-level multigrid: Krylov iterations and seconds of FP64 solves, plain vs multigrid",
           "value": float(np.mean(ratios)),
           "unit": "x (iterations plain / multigrid, mean over the operators with a plain arm)",
           "higher_is_better": True, "n_gpus": 1, "steps": 1, "warmup": 1, "data": "synthetic",
           "config": {"workload": "multigrid: %s; one Gaussian right-hand side each, FP64 to 1e-10"
                                  % "; ".join("%s %s" % (r["operator"], "x".join(map(str, r["lattice"]))) for r in rows)},
           "cases": rows}
    print(json.dumps(out), flush=True)


def oracle_sample(W, seconds, worker=0, n_workers=1):
    """The oracle as it stands, on a bounded sample of the workload: probes of
    one colouring (set 0, then further sets; worker w of n takes every n-th
    (set, colour) pair) solved one by one with its FP64 CG to 1e-10 and
    contracted; for Wilson, whose oracle solves take minutes, its operator
    applications on one probe.  Returns (site*RHS done, RHS count, seconds)."""
    import oracle.estimator as OE
    from oracle.colouring import greedy_colour
    from oracle.lattice import displace
    from oracle.probes import probe
    p, k = (4, 1) if W.kind == "lap" else W.pk[-1]
    col, m = greedy_colour(W.dims, W.mu, [p], k, 0)
    if W.kind == "lap":
        op = OE.Laplacian(W.dims, W.m2)
        kind, comps, applies = 0, [0], 1
    else:
        from paper_2106_01275_gb300 import inputs
        if W.csw:
            import oracle.clover as CL
            op = CL.WilsonClover(W.dims, inputs.gauge_links(W.dims, W.link_seed), W.kappa, W.csw, True)
        else:
            op = OE.Wilson(W.dims, inputs.gauge_links(W.dims, W.link_seed), W.kappa, True)
        kind, comps, applies = 1, list(range(12)), 2
    t0 = time.perf_counter()
    site_rhs, n_rhs = 0, 0
    if W.kind == "wil":
        v = probe(col, worker % m, SEED, 0, kind, op.dof, 0)
        while time.perf_counter() - t0 < seconds:
            v = op.apply(v) / 4.0
            site_rhs += W.N
            n_rhs += 1
        return site_rhs, n_rhs, time.perf_counter() - t0
    pair = 0
    while time.perf_counter() - t0 < seconds:
        s, c = divmod(pair, m)
        pair += 1
        if (pair - 1) % n_workers != worker:
            continue
        for a in comps:
            v = probe(col, c, SEED, s, kind, op.dof, a)
            x, its, rel = op.solve(v, TOL, MAXIT)
            _ = [np.vdot(v, displace(x, W.dims, W.mu, q)) for q in W.p_contract]
            site_rhs += (applies * its + 1) * W.N
            n_rhs += 1
    return site_rhs, n_rhs, time.perf_counter() - t0


def _oracle_worker(job):
    W, seconds, worker, n_workers = job
    return oracle_sample(W, seconds, worker, n_workers)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


class OraclePool:
    """The oracle on every host core: one spawned process per core (spawned,
    not forked, so that no CUDA state is inherited), each on its own share of
    the sample; numpy is kept to one thread per process."""

    def __init__(self, W):
        import multiprocessing as mp
        self.W = W
        self.n = os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.n)
        self.run(0.2)                                     # imports and first solves, untimed

    def run(self, seconds):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(self.W, seconds, w, self.n) for w in range(self.n)])
        wall = time.perf_counter() - t0
        return sum(r[0] for r in res), sum(r[1] for r in res), wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(W, seconds):
    pool = OraclePool(W)
    try:
        site, n_rhs, dt = pool.run(seconds)
    finally:
        pool.close()
    what = ("%d RHS of one colouring of %s, FP64 CG to 1e-10 with contraction" % (n_rhs, W.name)
            if W.kind == "lap" else "%d FP64 %s operator applications on %s"
            % (n_rhs, "clover Wilson" if W.csw else "Wilson", W.name))
    return {"value": site / dt, "unit": "site*RHS/s", "cores": pool.n, "kind": "oracle", "cpu_model": cpu_model(),
            "nproc": os.cpu_count(),
            "sample": "%s, %.1f s wall on %d processes (one per core)" % (what, dt, pool.n)}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    if args.workload == "grad32":
        dims = [16, 16, 16, 32] if args.case == "small" else [32, 32, 32, 64]
        W = Workload("grad32", "wil", dims, 2, [(4, 2)], [4], 1, "z4", "grad32 (oracle operator applications)",
                     kappa=0.12, link_seed=4321)
    else:
        W = workloads(args.case)[args.workload]
    per_step = max(2.0, min(20.0, args.cpu_seconds / max(args.steps, 1)))
    pool = OraclePool(W)
    try:
        for _ in range(args.warmup):
            pool.run(min(per_step, 2.0))
        t0 = time.perf_counter()
        site, n_rhs = 0.0, 0
        for _ in range(args.steps):
            sr, n, _ = pool.run(per_step)
            site += sr
            n_rhs += n
        t = time.perf_counter() - t0
    finally:
        pool.close()
    value = site / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site*RHS/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": W.desc + " (CPU oracle on a bounded sample per step)", "lattice": W.dims},
           "cpu_baseline": {"value": value, "unit": "site*RHS/s", "cores": pool.n, "kind": "oracle",
                            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                            "sample": ("%d %s over %d steps of %.1f s on %d processes (one per core)"
                                       % (n_rhs, "RHS solved and contracted" if W.kind == "lap" else
                                          "FP64 %s operator applications" % ("clover Wilson" if W.csw else "Wilson"),
                                          args.steps, per_step, pool.n))},
           "e2e": {"value": value, "unit": "site*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lap16", choices=["lap16", "wilson24", "clover24", "grad32", "colour", "deflation", "evenodd",
                                                        "multigrid"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-baselines", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="use the engine's default parameters")
    ap.add_argument("--tuning", default="", help="engine parameters fixed after tuning, e.g. rhs_block=8,cta_threads=256")
    ap.add_argument("--prec", default="mixed_fp32", choices=["mixed_fp32", "mixed_bf16"],
                    help="inner Krylov storage: FP32, or BF16 (FP32 arithmetic); FP64 outer either way")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: one colouring and few right-hand sides (for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "grad32":
        run_grad(args)
    elif args.workload == "colour":
        run_colour(args)
    elif args.workload == "deflation":
        run_deflation(args)
    elif args.workload == "evenodd":
        run_evenodd(args)
    elif args.workload == "multigrid":
        run_multigrid(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
