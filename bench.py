#!/usr/bin/env python3
"""Benchmark: all-at-once solves/sec on one GB300 (or N replicas).

One step = one full solve of script-A x = b (Eq. 1) to explicit relative
residual 1e-8 by right-preconditioned FGMRES with the nested-Chebyshev
alpha-circulant preconditioner, on the 2D 1024 x 1024 lognormal-diffusivity
workload (N = 1,048,576, ell = 10, alpha = 1e-2), complex-FP32 inner sweeps
with p = 40 Chebyshev steps per frequency and FP64 outer solve.  The all-FP64
GPU path is timed beside it on the same workload.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank solves its
own replica of the workload (the method has no cross-instance exchange):
weak scaling, value = total solves / max-over-ranks time.

--impl reference times the CPU oracle (oracle/, numpy FP64) instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("all-at-once solves/sec at rel. residual 1e-8 (mixed vs FP64 GPU); "
          "fused Chebyshev HBM GB/s")
UNIT = "solves/s"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    # name: (builder kwargs, p)
    "2d1024_p40": dict(n=1024, p=40, seed_field=21, seed_b=22),
    "2d1024_p10": dict(n=1024, p=10, seed_field=21, seed_b=22),
    "2d256_p20": dict(n=256, p=20, seed_field=11, seed_b=12),
}


def workload_name(w):
    d = WORKLOADS[w]
    return "2d_lognormal_%dx%d_l10_a1e-2_p%d" % (d["n"], d["n"], d["p"])


def make_problem(w):
    from paper_2506_03947_gb300 import inputs
    d = WORKLOADS[w]
    return inputs.config_2d(n=d["n"], ell=10, alpha=1e-2, inner_its=d["p"],
                            seed_field=d["seed_field"], seed_b=d["seed_b"])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Replicas:
    """The N > 1 path: one process per GPU, each solving its own replica of the workload.  The
    method has no exchange between instances, so the only collectives are a barrier around each
    timed region and the maximum of the timed durations; rank 0 alone prints."""

    def __init__(self, backend: str):
        self.rank, self.world, self.local = dist_env()
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v: float, device: str = "cpu") -> float:
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kind="tma"):
    """Hash of a fused-sweep kernel's source: its translation unit and the shared definitions it
    compiles against (grid descriptor, step tables, tile constants, TMA map, stream config)."""
    import re
    csrc = os.path.join(ROOT, "paper_2506_03947_gb300", "csrc")
    h = hashlib.sha256()
    unit = {"tma": "cheb_quad_tma.cu", "stream": "cheb_stream.cu", "tile": "cheb_d2.cu"}[kind]
    with open(os.path.join(csrc, unit), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(csrc, "aao_internal.cuh")) as fh:
        hdr = fh.read()
    pats = [r"struct GridDesc \{.*?\};", r"struct StepArgs \{.*?\};", r"struct QuadSteps \{.*?\};",
            r"struct alignas\(64\) FieldMap \{.*?\};", r"constexpr int kQuadTmaTY = \d+;",
            r"constexpr int kQuadTmaR = \d+;", r"constexpr long long kQuadTmaWaitCycles = [^;]*;",
            r"constexpr int kMaxEll = \d+;"]
    if kind == "stream":
        pats = [r"struct GridDesc \{.*?\};", r"struct StepArgs \{.*?\};", r"constexpr int kMaxFuse = \d+;",
                r"struct FuseSteps \{.*?\};", r"struct StreamConfig \{.*?\};", r"constexpr int kMaxEll = \d+;"]
    for pat in pats:
        m = re.search(pat, hdr, re.S)
        h.update((m.group(0) if m else pat).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key, kind="tma"):
    """dram bytes per launch from profiles/ncu_traffic.txt if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash(kind)
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if len(line) >= 3 and line[0] == kernel_key and line[1] == cur:
                return float(line[2])
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="aao_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi's start-up (its first query) can stall CUDA calls for tens of ms: wait for the
        # first sample so that it falls before the timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2506_03947_gb300 import binding
    from paper_2506_03947_gb300 import build as pkg_build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rep = Replicas("nccl")
    pkg_build.build()
    binding.load_library()

    def barrier():
        rep.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return rep.max(v, device="cuda")

    P = make_problem(args.workload)
    p = WORKLOADS[args.workload]["p"]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    kx = torch.from_numpy(P.kx.ravel()).cuda()
    ky = torch.from_numpy(P.ky.ravel()).cuda()
    b = torch.from_numpy(P.b).cuda()
    x = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    L = P.ell * P.N

    def timed_solves(solver, steps, warmup, profile=False, sampler=None):
        if sampler:
            sampler.start()                     # before the warm-up: its start-up is not timed
        for _ in range(warmup):
            solver.solve(b, x, P.tol, 64)
        barrier()
        if profile:
            solver.profile_enable(True)
        n0 = binding.aao_kernel_launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = time.perf_counter()
        walls = []
        for k in range(steps):
            flush.add_(1.0)                     # evict L2 between timed steps (not timed)
            ev[k][0].record(stream)
            tw = time.perf_counter()
            solver.solve(b, x, P.tol, 64)
            walls.append(time.perf_counter() - tw)
            ev[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
        timed_solves.walls = walls
        clocks = sampler.stop() if sampler else None
        launches = binding.aao_kernel_launch_count() - n0
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        prof = solver.profile() if profile else None
        if profile:
            solver.profile_enable(False)
        return ms, wall, launches, prof, clocks, solver.stats()

    # --- mixed precision (headline) ---
    s32 = binding.Solver(P.dim, P.n, kx, ky, None, P.ell, P.alpha, prec=binding.AAO_MIXED, inner_its=p,
                         restart=64, stream=sptr)
    sampler = ClockSampler(local) if not args.no_clocks else None
    # the fused sweep's kernel and launch configuration, chosen by the library's autotuner
    # (untimed: whole preconditioner applies per candidate, before any timed solve)
    tune_top = tail_top = None
    if not args.no_tune:
        _, cands = s32.autotune(3)
        tune_top = sorted((c for c in cands if not c["tail"]), key=lambda c: c["us_per_apply"])[:6]
        tail_top = sorted((c for c in cands if c["tail"]), key=lambda c: c["us_per_apply"])[:3]
    tuning = s32.tuning()
    tuning["tail"] = s32.stream_tail()
    quad_kind = s32.step_kernel()
    # timed solves run as the library runs them by default (each Arnoldi step replayed from
    # its CUDA graph); the per-kernel-class breakdown comes from a separate profiled pass,
    # where every class is bracketed by CUDA events on the launching stream
    ms, wall, launches, _, clocks, st32 = timed_solves(s32, args.steps, args.warmup, profile=False,
                                                       sampler=sampler)
    walls32 = list(timed_solves.walls)
    ms_max = max_over_ranks(ms)
    value = job_rate(world, args.steps, ms_max / 1e3)
    x32 = x.clone()
    prof_steps = max(3, args.steps // 2)
    ms_prof, _, _, prof, _, _ = timed_solves(s32, prof_steps, 1, profile=True)

    # --- end to end through the C ABI with pinned host buffers (copies timed) ---
    bh = torch.from_numpy(P.b).pin_memory()
    xh = torch.zeros(P.b.shape, dtype=torch.float64).pin_memory()
    for _ in range(max(1, min(args.warmup, 2))):
        s32.solve(bh, xh, P.tol, 64)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.add_(1.0)
        s32.solve(bh, xh, P.tol, 64)           # H2D b, solve, D2H x, stream synchronised
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = job_rate(world, args.steps, e2e_s)

    # --- all-FP64 GPU path on the same workload ---
    fp64 = None
    if not args.no_fp64:
        s32.close()
        s64 = binding.Solver(P.dim, P.n, kx, ky, None, P.ell, P.alpha, prec=binding.AAO_FP64, inner_its=p,
                             restart=64, stream=sptr)
        k64 = max(2, args.steps // 2)
        ms64, _, _, prof64, _, st64 = timed_solves(s64, k64, 1, profile=True)
        ms64 = max_over_ranks(ms64)
        rel = float(torch.linalg.norm(x - x32) / torch.linalg.norm(x))
        fp64 = {"value": job_rate(world, k64, ms64 / 1e3), "ms_per_step": ms64 / k64, "steps": k64,
                "outer_its": st64["outer_its"], "resid_explicit": st64["resid_explicit"],
                "mixed_vs_fp64_rel_diff": rel,
                "step_mid_gbs": (prof64["step_mid"]["bytes"] / (prof64["step_mid"]["ms"] * 1e-3) / 1e9
                                 if prof64["step_mid"]["ms"] > 0 else None)}
        s64.close()
    else:
        s32.close()

    # --- roofline of the dominant kernel (the fused Chebyshev sweep class with the most time)
    peak, peak_src = measured_peaks()
    sweep_classes = [k for k in ("step_quad", "step_pair", "step_mid") if prof[k]["launches"] > 0]
    dom = max(sweep_classes, key=lambda k: prof[k]["ms"])
    mid = prof[dom]
    per_launch_bytes = mid["bytes"] / max(1, mid["launches"])
    avg_ms = mid["ms"] / max(1, mid["launches"])
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    total_ms_prof = sum(v["ms"] for v in prof.values())
    quad_names = {binding.AAO_STEP_TMA: "k_cheb_quad_tma<10,2,2> (four fused multi-frequency Chebyshev steps, "
                                        "FP32, persistent, TMA-fed)",
                  binding.AAO_STEP_TILE: "k_cheb_quad<10,16,2> (four fused multi-frequency Chebyshev steps, FP32, "
                                         "shared-memory tile)",
                  binding.AAO_STEP_STREAM: "k_cheb_stream<S=%d,D=%d,NW=%d> (%d fused multi-frequency Chebyshev "
                                           "steps, FP32x2, warp strips streamed along y, H=%d, cp.async rings)"
                                           % (tuning["S"], tuning["D"], tuning["NW"], tuning["S"], tuning["H"])}
    kernels = {"step_quad": quad_names[quad_kind],
               "step_pair": "k_cheb_pair_v4<10,2> (two fused multi-frequency Chebyshev steps, FP32)",
               "step_mid": "k_cheb_step_v4<10,2,1,2,false> (fused multi-frequency Chebyshev step, FP32)"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": ncu_traffic(dom + "_" + args.workload, binding.KERNEL_NAMES.get(quad_kind, "tma")),
                "kernel": kernels[dom], "class": dom,
                "bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
                "launches": mid["launches"], "peak_source": peak_src + " hbm_gbs",
                "share_of_profiled_time": mid["ms"] / total_ms_prof if total_ms_prof > 0 else None,
                "profile_pass": {"steps": prof_steps, "ms_per_step": ms_prof / prof_steps,
                                 "note": "kernel classes timed by CUDA events in separate solves, without graphs"},
                "classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else None)}
                            for k, v in prof.items()}}

    batch = None
    if not args.no_batch:
        batch = run_batch_leg(args, binding, torch, sptr, peak)
    rhs3d = None
    if not args.no_rhs3d:
        rhs3d = run_rhs3d_leg(args, binding, torch, sptr, peak)
    best = None
    if not args.no_best_case:
        best = run_best_case_leg(args, binding, torch, sptr)
    sweep = None
    if not args.no_sweep:
        sweep = run_sweep_leg(args, binding, torch, sptr)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args.workload, P, p, st32["outer_its"])

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 inner / f64 outer",
        "data": "synthetic (seeded lognormal diffusivity, b_1 ~ N(0,1))",
        "config": bench_config(args.workload, P, p, world), "precision": "mixed",
        "outer_its": st32["outer_its"], "resid_explicit": st32["resid_explicit"],
        "a_matvecs": st32["a_matvecs"], "wall_ms_per_step": wall * 1e3 / args.steps,
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * L, "d2h_bytes_per_step": 8 * L},
        "gpu_launches": launches, "clocks": clocks, "fp64_gpu": fp64, "batch": batch, "rhs3d": rhs3d, "best_case": best,
        "sweep": sweep, "step_wall_ms": [round(w * 1e3, 3) for w in walls32],
        "fused_sweep": {"tuning": tuning, "fastest_candidates": tune_top,
                        "fastest_tail_candidates": tail_top},
    }
    # compact summary last, so that a truncated capture of the line still carries it
    out["headline"] = {
        "mixed_solves_s": round(value, 3), "e2e_solves_s": round(e2e_value, 3),
        "fp64_solves_s": round(fp64["value"], 3) if fp64 else None,
        "outer_its_mixed": st32["outer_its"], "outer_its_fp64": fp64["outer_its"] if fp64 else None,
        "mixed_vs_fp64_rel_diff": fp64["mixed_vs_fp64_rel_diff"] if fp64 else None,
        "fused_kernel": binding.KERNEL_NAMES.get(quad_kind), "fused_us_per_launch": round(avg_ms * 1e3, 2),
        "roofline_frac": round(achieved / peak, 4),
        "batch_instance_solves_s": round(batch["value"], 2) if batch else None,
        "batch_fp64_sequential_solves_s": round(batch["fp64_sequential"]["value"], 2) if batch else None,
        "rhs3d_rhs_solves_s": round(rhs3d["value"], 3) if rhs3d else None,
        "cpu_oracle_solves_s": cpu["value"] if cpu else None}
    if rank == 0:
        print(json.dumps(out), flush=True)
    rep.close()


def run_batch_leg(args, binding, torch, sptr, peak):
    """Batched workload: 64 instances, grids from {128..512}^2, ell in {6..12}, alpha in {1e-1, 1e-2},
    per-instance lognormal diffusivity (sigma ~ U[0.2, 1]), p = 20, tol 1e-8, all solved in one
    lockstep batch (one launch per phase, CUDA graph per Arnoldi step) and, for comparison, one
    after another with single-instance handles."""
    from paper_2506_03947_gb300 import inputs
    probs = inputs.config_batch(count=args.batch_count)
    solvers = [binding.Solver(P.dim, P.n, P.kx.ravel(), P.ky.ravel(), None, P.ell, P.alpha,
                              prec=binding.AAO_MIXED, inner_its=P.inner_its, restart=64, stream=sptr)
               for P in probs]
    bs = [torch.from_numpy(P.b).cuda() for P in probs]
    xs = [torch.zeros_like(v) for v in bs]
    bat = binding.Batch(solvers, use_graphs=True)
    for _ in range(2):
        bat.solve(bs, xs, 1e-8, 200)
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        bat.solve(bs, xs, 1e-8, 200)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / reps
    its = [bat.stats(i)["outer_its"] for i in range(len(probs))]
    conv = all(bat.stats(i)["converged"] for i in range(len(probs)))
    # the fused sweeps' bandwidth: one more solve with event timing of those launches (no graphs)
    bat.profile_enable(True)
    bat.solve(bs, xs, 1e-8, 200)
    bprof = bat.profile()
    bat.profile_enable(False)
    fused_gbs = bprof["bytes"] / (bprof["ms"] * 1e-3) / 1e9 if bprof["ms"] > 0 else None
    xb = [v.clone() for v in xs]              # the batch's solutions
    # sequential reference: the same instances one after another (single-instance path)
    for s, b, x in zip(solvers, bs, xs):
        s.solve(b, x, 1e-8, 200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, b, x in zip(solvers, bs, xs):
        s.solve(b, x, 1e-8, 200)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    bat.close()
    # the all-FP64 GPU form of the same instances, one after another (a handle per instance,
    # created and destroyed outside the timed solves), for the comparison at equal accuracy
    t64 = 0.0
    its64, diff64 = [], []
    for s, P, b, xm in zip(solvers, probs, bs, xb):
        s64 = binding.Solver(P.dim, P.n, P.kx.ravel(), P.ky.ravel(), None, P.ell, P.alpha, prec=binding.AAO_FP64,
                             inner_its=P.inner_its, restart=64, stream=sptr)
        x64 = torch.zeros_like(b)
        s64.solve(b, x64, 1e-8, 200)
        torch.cuda.synchronize()
        x64.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        s64.solve(b, x64, 1e-8, 200)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1) * 1e-3
        its64.append(s64.stats()["outer_its"])
        diff64.append(float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)))
        s64.close()
    cells = sum(P.N * P.ell for P in probs)
    return {"workload": "%d instances, grids {128..512}^2, ell {6..12}, alpha {1e-1,1e-2}, p=20, tol 1e-8"
                        % len(probs),
            "instances": len(probs), "ell_N_total": cells,
            "value": len(probs) / tb, "unit": "instance solves/s", "ms_per_batch": tb * 1e3,
            "sequential_value": len(probs) / ts, "sequential_ms": ts * 1e3,
            "outer_its_max": max(its), "outer_its_mean": sum(its) / len(its), "all_converged": conv,
            "fp64_sequential": {"value": len(probs) / t64, "unit": "instance solves/s", "ms": t64 * 1e3,
                                "outer_its_max": max(its64), "outer_its_mean": sum(its64) / len(its64),
                                "batch_minus_fp64_its_max": max(a - b for a, b in zip(its, its64)),
                                "batch_vs_fp64_rel_diff_max": max(diff64),
                                "timing": "CUDA events around one solve per instance (after one untimed solve), "
                                          "all-FP64 handles one after another"},
            "fused_sweep": {"kernel": "kb_cheb_stream<S=4,D=3,NW=8> and the final kb_cheb_stream<S=2,D=3,NW=8> "
                                      "(persistent warp-strip launches over (member, frequency pair, segment, "
                                      "strip) units from a device queue)",
                            "launches": bprof["launches"], "avg_launch_ms": bprof["ms"] / max(1, bprof["launches"]),
                            "bytes_per_launch": bprof["bytes"] / max(1, bprof["launches"]),
                            "achieved_gbs": fused_gbs, "peak_gbs": peak,
                            "frac": (fused_gbs / peak if fused_gbs else None),
                            "timing": "CUDA events around the back-to-back fused launches of each Arnoldi step in one extra solve without graphs"},
            "timing": "host wall clock around synchronised batch solves (3 reps after 2 warm-ups)"}


def run_rhs3d_leg(args, binding, torch, sptr, peak):
    """3D multi-right-hand-side workload: 128^3 cells, ell = 10, alpha = 1e-2, anisotropic lognormal
    diffusivity (sigma 0.7, correlation lengths 8/8/4), p = 15, eight right-hand sides solved
    together (aao_solve_multi: lockstep views of one handle sharing its operator) and, for
    comparison, one after another on one handle (mixed precision, tol 1e-8), inputs resident on the
    device.  Reports right-hand-side solves per second and the bandwidth of the 3D Chebyshev step."""
    from paper_2506_03947_gb300 import inputs
    P = inputs.config_3d()
    kx = torch.from_numpy(P.kx.ravel()).cuda()
    ky = torch.from_numpy(P.ky.ravel()).cuda()
    kz = torch.from_numpy(P.kz.ravel()).cuda()
    s = binding.Solver(3, P.n, kx, ky, kz, P.ell, P.alpha, prec=binding.AAO_MIXED, inner_its=P.inner_its,
                       restart=64, stream=sptr)
    bs = [torch.from_numpy(P.b[i]).cuda() for i in range(P.b.shape[0])]
    x = torch.zeros_like(bs[0])
    s.solve(bs[0], x, P.tol, 64)                 # warm-up
    torch.cuda.synchronize()
    # the eight right-hand sides together (aao_solve_multi): one untimed call allocates the views
    xs = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xs, P.tol, 64)
    torch.cuda.synchronize()
    for v in xs:
        v.zero_()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(torch.cuda.current_stream())
    s.solve_multi(bs, xs, P.tol, 64)
    m1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms_multi = m0.elapsed_time(m1)
    its_multi = [s.multi_stats(i)["outer_its"] for i in range(len(bs))]
    res_multi = [s.multi_stats(i)["resid_explicit"] for i in range(len(bs))]
    # the shared-stencil step's bandwidth: one more multi solve with event timing of the middle
    # Chebyshev steps (no graphs)
    s.multi_profile_enable(True)
    for v in xs:
        v.zero_()
    s.solve_multi(bs, xs, P.tol, 64)
    mprof = s.multi_profile()
    s.multi_profile_enable(False)
    mgbs = mprof["bytes"] / (mprof["ms"] * 1e-3) / 1e9 if mprof["ms"] > 0 else None
    s.close()
    del xs
    s = binding.Solver(3, P.n, kx, ky, kz, P.ell, P.alpha, prec=binding.AAO_MIXED, inner_its=P.inner_its,
                       restart=64, stream=sptr)
    s.solve(bs[0], x, P.tol, 64)                 # warm-up
    torch.cuda.synchronize()
    s.profile_enable(True)
    its, res = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    for b in bs:
        x.zero_()
        s.solve(b, x, P.tol, 64)
        st = s.stats()
        its.append(st["outer_its"])
        res.append(st["resid_explicit"])
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.profile_enable(False)
    s.close()
    sweep = prof["step_mid"]
    sweep_gbs = sweep["bytes"] / (sweep["ms"] * 1e-3) / 1e9 if sweep["ms"] > 0 else None
    total = sum(v["ms"] for v in prof.values())
    return {"workload": "3d_lognormal_128^3_l10_a1e-2_p15_x8rhs", "rhs": len(bs),
            "value": len(bs) / (ms_multi * 1e-3), "unit": "rhs solves/s", "ms_per_rhs": ms_multi / len(bs),
            "multi": {"outer_its": its_multi, "resid_explicit_max": max(res_multi),
                      "all_converged": all(r < P.tol for r in res_multi),
                      "timing": "CUDA events around one aao_solve_multi of the 8 right-hand sides (views allocated by "
                                "an untimed call before)",
                      "sweep": {"kernel": "kb_step_shared<10,3,1,2> (one Chebyshev step of every right-hand "
                                          "side per launch; each tile's stencil loaded once)",
                                "launches": mprof["launches"],
                                "avg_launch_ms": mprof["ms"] / max(1, mprof["launches"]),
                                "bytes_per_launch": mprof["bytes"] / max(1, mprof["launches"]),
                                "achieved_gbs": mgbs, "peak_gbs": peak,
                                "frac": (mgbs / peak if mgbs else None),
                                "timing": "CUDA events around the steps 2 .. p-1 of each Arnoldi step in one "
                                          "extra solve without graphs"}},
            "one_after_another": {"value": len(bs) / (ms * 1e-3), "ms_per_rhs": ms / len(bs)},
            "outer_its": its, "resid_explicit_max": max(res), "all_converged": all(r < P.tol for r in res),
            "sweep_kernel": "k_cheb_step_v4<10,3,1,2,false> (one multi-frequency Chebyshev step, FP32, 7-point)",
            "sweep_gbs": sweep_gbs, "sweep_frac": (sweep_gbs / peak if sweep_gbs else None),
            "sweep_bytes_per_cell": 16 * P.ell + 12,
            "share": {k: round(v["ms"] / total, 3) for k, v in prof.items() if v["ms"] > 0},
            "timing": "CUDA events around 8 device-resident solves after one warm-up solve"}


def run_best_case_leg(args, binding, torch, sptr):
    """Outer iterations of P_NC (p = 40, 10) and P_SP (10 Krylov steps per shifted solve) against
    the paper's best-case P_alpha (applied exactly through the spatial DCT, FP64) on a
    constant-diffusivity grid (kappa = 50/ell on every face), 256^2, ell = 10, tol 1e-8, over
    alpha; plus the time of one best-case solve at 1024^2."""
    import numpy as np
    from paper_2506_03947_gb300 import inputs
    rows = []
    for alpha in (1e-1, 1e-2, 1e-3, 1e-4):
        P = inputs.make_problem("const256", 2, (256, 256), 10, alpha, 1, 0.0, (16.0, 16.0), 41, 42)
        kx = torch.from_numpy(P.kx.ravel()).cuda()
        ky = torch.from_numpy(P.ky.ravel()).cuda()
        b = torch.from_numpy(P.b).cuda()
        row = {"alpha": alpha}
        for name, prec, p, mode in (("best_case", binding.AAO_FP64, 1, binding.AAO_PRECOND_EXACT_DCT),
                                    ("nc_p40", binding.AAO_MIXED, 40, binding.AAO_PRECOND_NC),
                                    ("nc_p10", binding.AAO_MIXED, 10, binding.AAO_PRECOND_NC),
                                    ("sp_k10", binding.AAO_FP64, 10, binding.AAO_PRECOND_SP)):
            s = binding.Solver(2, P.n, kx, ky, None, P.ell, alpha, prec=prec, inner_its=p, restart=64, stream=sptr)
            if mode != binding.AAO_PRECOND_NC:
                s.set_precond_mode(mode)
            x = torch.zeros_like(b)
            s.solve(b, x, 1e-8, 64, allow_notconv=True)
            row[name] = s.stats()["outer_its"]
            s.close()
        rows.append(row)
    P = inputs.make_problem("const1024", 2, (1024, 1024), 10, 1e-2, 1, 0.0, (16.0, 16.0), 21, 22)
    kx = torch.from_numpy(P.kx.ravel()).cuda()
    ky = torch.from_numpy(P.ky.ravel()).cuda()
    b = torch.from_numpy(P.b).cuda()
    s = binding.Solver(2, P.n, kx, ky, None, P.ell, P.alpha, prec=binding.AAO_FP64, inner_its=1, restart=64,
                       stream=sptr)
    s.set_precond_mode(binding.AAO_PRECOND_EXACT_DCT)
    x = torch.zeros_like(b)
    s.solve(b, x, 1e-8, 64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    x.zero_()
    e0.record(torch.cuda.current_stream())
    s.solve(b, x, 1e-8, 64)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    its1024 = s.stats()["outer_its"]
    s.close()
    return {"workload": "2d_const_256x256_l10 (kappa 5), tol 1e-8; outer iterations",
            "alpha_sweep": rows,
            "best_case_1024": {"alpha": 1e-2, "outer_its": its1024, "ms_per_solve": e0.elapsed_time(e1),
                               "note": "FP64, spatial DCT by the library's own FFT-based kernels (power-of-two axes)"}}


def run_sweep_leg(args, binding, torch, sptr):
    """Outer iterations and time per solve, mixed and FP64, tol 1e-8, restart 64: over alpha in
    {1e-1, 1e-2, 1e-3} and p in {10, 20, 40} on the lognormal 256^2 grid (sigma 0.5, correlation
    length 16, seeds 11/12, L2-resident), and at p = 10 on the 1024^2 grid of the main workload.
    Each solve runs once untimed (graph capture), then once timed by CUDA events."""
    from paper_2506_03947_gb300 import inputs

    def timed(P, prec, p):
        kx = torch.from_numpy(P.kx.ravel()).cuda()
        ky = torch.from_numpy(P.ky.ravel()).cuda()
        b = torch.from_numpy(P.b).cuda()
        s = binding.Solver(2, P.n, kx, ky, None, P.ell, P.alpha, prec=prec, inner_its=p, restart=64, stream=sptr)
        x = torch.zeros_like(b)
        s.solve(b, x, 1e-8, 64, allow_notconv=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        x.zero_()
        e0.record(torch.cuda.current_stream())
        s.solve(b, x, 1e-8, 64, allow_notconv=True)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        st = s.stats()
        s.close()
        return {"outer_its": st["outer_its"], "ms_per_solve": round(e0.elapsed_time(e1), 3),
                "resid_explicit": st["resid_explicit"], "converged": bool(st["converged"])}

    rows = []
    for alpha in (1e-1, 1e-2, 1e-3):
        P = inputs.config_2d(n=256, alpha=alpha, seed_field=11, seed_b=12)
        for p in (10, 20, 40):
            rows.append({"alpha": alpha, "p": p, "mixed": timed(P, binding.AAO_MIXED, p),
                         "fp64": timed(P, binding.AAO_FP64, p)})
    P = inputs.config_2d(n=1024, alpha=1e-2, seed_field=21, seed_b=22)
    big = {"mixed": timed(P, binding.AAO_MIXED, 10), "fp64": timed(P, binding.AAO_FP64, 10)}
    return {"workload": "2d_lognormal_256x256_l10 (sigma 0.5, corr 16, seeds 11/12), tol 1e-8",
            "grid256": rows, "grid1024_a1e-2_p10": big}


def run_ncu_case(args):
    """Small launch sequence for ncu captures: preconditioner applies only.

    The workload's grid and coefficients, a solver with a one-vector Krylov
    space (so the device holds about 1 GB), and --steps applications of
    P_NC^{-1} (one transform, p Chebyshev steps each).
    """
    import torch

    from paper_2506_03947_gb300 import binding
    from paper_2506_03947_gb300 import build as pkg_build
    pkg_build.build()
    P = make_problem(args.workload)
    p = WORKLOADS[args.workload]["p"]
    prec = binding.AAO_FP64 if args.ncu_fp64 else binding.AAO_MIXED
    sptr = torch.cuda.current_stream().cuda_stream
    s = binding.Solver(P.dim, P.n, P.kx.ravel(), P.ky.ravel(), None, P.ell, P.alpha, prec=prec, inner_its=p,
                       restart=1, stream=sptr)
    if args.step_kernel != "auto":
        s.set_step_kernel({"tile": binding.AAO_STEP_TILE, "tma": binding.AAO_STEP_TMA,
                           "stream": binding.AAO_STEP_STREAM}[args.step_kernel])
    if args.stream_config:
        s.set_stream_config(*[int(v) for v in args.stream_config.split(",")])
    r = torch.from_numpy(P.b).cuda()
    z = torch.empty_like(r)
    for _ in range(args.steps):
        s.precond_apply(r, z)
    torch.cuda.synchronize()
    if args.ncu_solve:
        s.close()
        s = binding.Solver(P.dim, P.n, P.kx.ravel(), P.ky.ravel(), None, P.ell, P.alpha, prec=prec,
                           inner_its=p, restart=16, stream=sptr)
        x = torch.zeros_like(r)
        s.solve(r, x, P.tol, 16, allow_notconv=True)
        torch.cuda.synchronize()
    print(json.dumps({"ncu_case": workload_name(args.workload), "prec": "fp64" if args.ncu_fp64 else "mixed",
                      "applies": args.steps, "launches": binding.aao_kernel_launch_count(),
                      "z_norm": float(torch.linalg.norm(z))}))


def run_ncu_batch(args):
    """One batched solve of the 64-instance workload with direct launches (no CUDA graphs), for
    an ncu launch list of the batch's kernels.  The device holds about 65 GB (Krylov spaces of
    restart 64); every launch is short."""
    import torch

    from paper_2506_03947_gb300 import binding
    from paper_2506_03947_gb300 import build as pkg_build
    from paper_2506_03947_gb300 import inputs
    pkg_build.build()
    probs = inputs.config_batch(count=args.batch_count)
    sptr = torch.cuda.current_stream().cuda_stream
    solvers = [binding.Solver(P.dim, P.n, P.kx.ravel(), P.ky.ravel(), None, P.ell, P.alpha,
                              prec=binding.AAO_MIXED, inner_its=P.inner_its, restart=64, stream=sptr)
               for P in probs]
    bs = [torch.from_numpy(P.b).cuda() for P in probs]
    xs = [torch.zeros_like(v) for v in bs]
    bat = binding.Batch(solvers, use_graphs=False)
    n0 = binding.aao_kernel_launch_count()
    bat.solve(bs, xs, 1e-8, 200)
    torch.cuda.synchronize()
    its = [bat.stats(i)["outer_its"] for i in range(len(probs))]
    print(json.dumps({"ncu_batch": len(probs), "launches": binding.aao_kernel_launch_count() - n0,
                      "outer_its_max": max(its), "outer_its_mean": sum(its) / len(its)}))


def run_ncu_multi(args):
    """One multi-right-hand-side solve (aao_solve_multi) of the 3D workload's operator at 96^3 with
    eight right-hand sides, for an ncu launch list of its kernels (about 80 GB on the device)."""
    import torch

    from paper_2506_03947_gb300 import binding
    from paper_2506_03947_gb300 import build as pkg_build
    from paper_2506_03947_gb300 import inputs
    pkg_build.build()
    P = inputs.config_3d(n=96)
    sptr = torch.cuda.current_stream().cuda_stream
    kx, ky, kz = (torch.from_numpy(a.ravel()).cuda() for a in (P.kx, P.ky, P.kz))
    s = binding.Solver(3, P.n, kx, ky, kz, P.ell, P.alpha, prec=binding.AAO_MIXED, inner_its=P.inner_its,
                       restart=64, stream=sptr)
    bs = [torch.from_numpy(P.b[i]).cuda() for i in range(P.b.shape[0])]
    xs = [torch.zeros_like(b) for b in bs]
    n0 = binding.aao_kernel_launch_count()
    s.solve_multi(bs, xs, P.tol, 64)
    torch.cuda.synchronize()
    its = [s.multi_stats(i)["outer_its"] for i in range(len(bs))]
    print(json.dumps({"ncu_multi": len(bs), "grid": list(P.n), "launches": binding.aao_kernel_launch_count() - n0,
                      "outer_its": its}))


def oracle_iterations(P, p, steps, warmup):
    """Time the oracle (numpy FP64) iteration by iteration on the full workload.

    The oracle solves the workload's system (FGMRES with P_NC, tol 1e-8, x_0 = 0) back to back,
    as many solves as it takes; every outer FGMRES iteration of that stream is one unit.  The
    first ``warmup`` iterations are untimed, the next ``steps`` are timed with the host clock
    (the work between two iterations - the solution update, the explicit residual and the next
    solve's first residual - falls into the next iteration's interval).  Returns the per-iteration
    durations and the outer iteration counts of the solves that finished.
    """
    from oracle import solve

    stamps = []
    finished = []

    class Enough(Exception):
        pass

    def tick(_):
        stamps.append(time.perf_counter())
        if len(stamps) > warmup + steps:
            raise Enough()

    stamps.append(time.perf_counter())
    try:
        while True:
            res = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, p, P.tol, 64, callback=tick)
            finished.append(res.outer_its)
    except Enough:
        pass
    t = stamps[warmup:warmup + steps + 1]
    return [b - a for a, b in zip(t[:-1], t[1:])], finished


def oracle_rate(durations, its_per_solve):
    """Solve-equivalents per second: timed iterations / (iterations per solve x their time)."""
    return len(durations) / (its_per_solve * sum(durations))


def oracle_sample_in_child(workload, p, threads, iters=3):
    """Durations of the first `iters` outer FGMRES iterations of an oracle solve, timed in a fresh
    Python process whose BLAS/OpenMP thread pools are set to `threads` before numpy loads (this
    process's numpy was loaded with the default pools) and which sees no GPU."""
    code = ("import json, bench; P = bench.make_problem(%r); "
            "d, _ = bench.oracle_iterations(P, %d, %d, 0); print(json.dumps(d))" % (workload, p, iters))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: %s" % r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_sample(workload, P, p, outer_its):
    """Oracle (numpy FP64) on a bounded sample: three consecutive outer FGMRES iterations of a
    real oracle solve of the full workload, converted to solves/s with the outer iteration count
    the solve needs; on one thread, and on all of the host's cores (BLAS pools; the oracle's
    sparse products and transforms stay single-threaded)."""
    nproc = os.cpu_count() or 1
    d1 = oracle_sample_in_child(workload, p, 1)
    dn = oracle_sample_in_child(workload, p, nproc)
    desc = "the first 3 outer FGMRES iterations of an oracle solve on the full %dx%d grid (%.2f s), over %d " \
           "outer iterations per solve"
    return {"value": oracle_rate(d1, outer_its), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": desc % (P.n[0], P.n[1], sum(d1), outer_its),
            "all_cores": {"value": oracle_rate(dn, outer_its), "unit": UNIT, "cores": nproc, "kind": "oracle",
                          "sample": desc % (P.n[0], P.n[1], sum(dn), outer_its) +
                          "; numpy's BLAS pools on all %d cores of this host" % nproc}}


def oracle_outer_its(workload):
    path = os.path.join(ROOT, "tests", "golden", "oracle_outer_its.txt")
    with open(path) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if parts and parts[0] == workload_name(workload):
                return int(parts[1])
    raise RuntimeError("no oracle iteration count for %s in %s" % (workload, path))


def bench_config(workload, P, p, world):
    """The workload description both arms print (identical dicts)."""
    return {"workload": workload_name(workload),
            "grid": [P.n[0], P.n[1]], "N": P.N, "ell": P.ell, "alpha": P.alpha, "inner_its": p,
            "tol": P.tol, "restart": 64,
            "l2": "working set above the 129 MB L2; the GPU arm also flushes L2 (256 MiB write) "
                  "between timed steps",
            "parallelism": "replicas" if world > 1 else "single device"}


def run_reference(args):
    """The oracle on the host cores, one thread (BLAS threads pinned to 1 before numpy loads).

    One step = one outer FGMRES iteration of back-to-back oracle solves of the full workload
    (measured, not extrapolated); value = solve-equivalents per second = steps / (outer
    iterations per solve x timed seconds), with the iteration count the oracle's own solves took
    in this run (from the golden file if no solve finished inside the run)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    P = make_problem(args.workload)
    p = WORKLOADS[args.workload]["p"]
    d, finished = oracle_iterations(P, p, args.steps, args.warmup)
    its = finished[0] if finished else oracle_outer_its(args.workload)
    value = oracle_rate(d, its)
    T = sum(d)
    sample = ("each step: one outer FGMRES iteration of back-to-back oracle solves of the full %dx%d grid "
              "(%d timed, mean %.2f s, after %d untimed); %d outer iterations per oracle solve (%s); "
              "solves finished in the run: %d" % (P.n[0], P.n[1], len(d), T / len(d), args.warmup, its,
                                                  "measured in this run" if finished else "golden file",
                                                  len(finished)))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": T * 1e3 / len(d),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded lognormal diffusivity, b_1 ~ N(0,1))",
           "config": bench_config(args.workload, P, p, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "oracle_ms_per_iteration": [round(v * 1e3, 1) for v in d]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="2d1024_p40")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (use the default fused sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-instance workload")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-rhs3d", action="store_true", help="skip the 3D 128^3 eight-right-hand-side workload")
    ap.add_argument("--no-best-case", action="store_true", help="skip the best-case (exact P_alpha) comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the alpha / p sweep (256^2) and the 1024^2 p = 10 solves")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run only preconditioner applies (small device footprint) for ncu captures")
    ap.add_argument("--ncu-fp64", action="store_true", help="with --ncu-case: FP64 path")
    ap.add_argument("--step-kernel", choices=["auto", "tile", "tma", "stream"], default="auto",
                    help="with --ncu-case: the fused-step kernel (shared-memory tile, persistent TMA or "
                         "warp-strip)")
    ap.add_argument("--stream-config", default="",
                    help="with --ncu-case: S,H,D,NW of the warp-strip kernel")
    ap.add_argument("--ncu-solve", action="store_true",
                    help="with --ncu-case: also one solve with a 16-vector Krylov space (about 3 GB)")
    ap.add_argument("--ncu-batch", action="store_true",
                    help="run only one batched solve of the 64-instance workload without graphs (ncu launch list)")
    ap.add_argument("--ncu-multi", action="store_true",
                    help="run only one eight-right-hand-side solve of the 3D operator at 96^3 (ncu launch list)")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.ncu_batch:
        run_ncu_batch(args)
        return
    if args.ncu_multi:
        run_ncu_multi(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
