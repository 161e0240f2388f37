"""Benchmark: second-order thin-disk force on the 4096^2 uniform grid, FP32.

One step = one full solve through the C ABI (restriction is empty on one
level; forward row pass with the slopes, column pass with the spectral
multiply-accumulate, inverse row pass), kernel spectra resident in HBM (built
once per shape at plan creation, timed separately as plan_ms).

Prints ONE JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
a bounded sample of the same workload instead.

Multi-GPU (torchrun): every rank solves its own replica of the workload; there
is no data-path collective (replicas only); the timed region is bracketed by a
barrier and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

N_DEFAULT = 4096
METRIC = "force cells/s"
UNIT = "cells/s"
L2_BYTES = 129 * 2 ** 20


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# Sources of the timed transform kernels: a change to any of them makes the
# recorded DRAM traffic stale.
KERNEL_SOURCES = ("sgf_kernels.cuh", "sgf_fft16.cuh", "sgf_fft.cuh", "sgf_tc.cuh", "sgf_internal.h",
                  "sgf_inst_12.cu")


def csrc_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        p = ROOT / "paper_1603_03142_gb300" / "csrc" / name
        h.update(name.encode())
        h.update(p.read_bytes())
    return h.hexdigest()


def recorded_ncu(kernel: str, table: str = "dram_bytes_per_launch"):
    """A per-launch ncu figure of `kernel` from the committed summary (DRAM
    bytes, or the FP32-pipe record), or None when the CUDA sources changed
    since those counters were taken."""
    f = ROOT / "profiles" / "traffic.json"
    if not f.exists():
        return None
    try:
        d = json.loads(f.read_text())
    except ValueError:
        return None
    if d.get("csrc_sha256") != csrc_digest():
        return None
    return d.get(table, {}).get(kernel)


def recorded_traffic(kernel: str):
    return recorded_ncu(kernel)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SGF_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def oracle_sample_rate(n: int, seconds: float = 12.0, seed: int = 0):
    """Oracle cells/s on a bounded sample of target cells of the 4096^2 workload."""
    import numpy as np
    import oracle
    from paper_1603_03142_gb300 import workloads as W
    nest, sigma = W.config3(n, seed=0)
    prepared = oracle.prepare(nest, sigma)
    rng = np.random.Generator(np.random.PCG64(seed))
    cores = oracle.max_threads()
    # calibrate with one target per core, then size the sample to ~`seconds`
    k0 = max(1, cores)
    ii = rng.integers(0, n, k0)
    jj = rng.integers(0, n, k0)
    t0 = time.perf_counter()
    oracle.force_at(nest, sigma, np.zeros(k0, dtype=int), ii, jj, prepared=prepared)
    dt0 = time.perf_counter() - t0
    k = max(k0, int(k0 * seconds / max(dt0, 1e-3)) // k0 * k0)
    ii = rng.integers(0, n, k)
    jj = rng.integers(0, n, k)
    t0 = time.perf_counter()
    oracle.force_at(nest, sigma, np.zeros(k, dtype=int), ii, jj, prepared=prepared)
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} seeded target cells of the {n}^2 grid, full direct sum over all {n * n} "
                      f"source cells each ({dt:.1f} s)", "seconds": dt, "targets": k}


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps = []
    for s in range(args.warmup + args.steps):
        warm = s < args.warmup
        info = oracle_sample_rate(args.n, seconds=1.0 if warm else args.ref_seconds, seed=s)
        if not warm:
            steps.append(info)
    tot_t = sum(x["seconds"] for x in steps)
    tot_c = sum(x["targets"] for x in steps)
    value = tot_c / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"uniform-{args.n}x{args.n}-lognormal-taper", "n": args.n, "levels": 1,
                       "precision": "fp32", "parallelism": "replicas", "engine": "cpu-fp64-oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": steps[-1]["cores"], "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_forest(args, world, dev, stream):
    """Example 3's geometry (Sec. 3: two disks, six level-0 tiles and two level-1
    patches of forest_n^2 cells each, the paper's N = 2 forest_n), FP32: ms per
    solve over rotating input/output sets larger than L2, and the plan's
    algorithmic bytes over that time."""
    import numpy as np
    import torch
    from paper_1603_03142_gb300 import sgf, workloads as W
    f = W.example3_forest(args.forest_n)
    sig0 = [torch.from_numpy(a.astype(np.float32)).to(dev) for a in W.two_disk_density(f)]
    plan = sgf.Plan(f, "fp32")
    plan.autotune(reps=3)
    per_set = 3 * sum(a.numel() for a in sig0) * 4
    sets = max(2, -(-4 * L2_BYTES // per_set))
    sig = [[a.roll(shifts=k, dims=1).contiguous() for a in sig0] for k in range(sets)]
    fx = [[torch.empty_like(a) for a in sig0] for _ in range(sets)]
    fy = [[torch.empty_like(a) for a in sig0] for _ in range(sets)]

    def step(k):
        plan.solve_ptrs([a.data_ptr() for a in sig[k % sets]], [a.data_ptr() for a in fx[k % sets]],
                        [a.data_ptr() for a in fy[k % sets]], stream)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    plan.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    plan.profile(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = plan.profile_read()
    st = plan.stats()
    cells = sum(a.numel() for a in sig0)
    out = {"workload": f"two-disk forest (Example 3): 6 level-0 + 2 level-1 patches of {args.forest_n}^2",
           "cells": cells, "cells_per_s": world * cells / (ms / 1e3), "ms_per_step": ms,
           "schedule": plan.schedule(), "launches_per_solve": st["launches_per_solve"],
           "spectra_mib": st["spectra_bytes"] / 2**20,
           "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in prof["kernels"].items() if v["launches"]},
           "algorithmic_bytes_per_solve": st["algorithmic_bytes"],
           "solve_gbs": st["algorithmic_bytes"] / (ms / 1e3) / 1e9,
           "solve_frac_of_peak": st["algorithmic_bytes"] / (ms / 1e3) / 1e9 / peaks()[0],
           "l2": f"{sets} rotating input/output sets ({sets * per_set / 2**20:.0f} MiB)"}
    plan.close()
    return out


def nest_pair_bytes(nests, w: int = 4):
    """Algorithmic HBM bytes of one solve of each nest (one patch per level, force
    plans, w bytes per real), split by pair of levels: the same accounting as the
    library's plan statistics (every intermediate written and read once, every
    kernel spectrum read once per use, padding not counted).  Case 1 carries the
    level's own forward slab and main output; a Case-2 pair (finer source, m =
    2^d) its m^2 phase slabs of n/m rows and m^2 phase spectra; a Case-3 pair
    (coarser source) its m^2 phase outputs of n/m rows and m^2 phase spectra:
    bytes grow with m for the intermediates and m^2 for the spectra."""
    C = 2 * w
    out = {}

    def add(key, b):
        out[key] = out.get(key, 0) + b
    for nest in nests:
        n, L = int(nest.n), int(nest.levels)
        n1 = n + 1
        add("sigma_in_forces_out", 3 * L * n * n * w)
        if L > 1:  # restriction of every covered level: its input, its copy, the children of its covered cells
            add("restriction", (L - 1) * (2 * n * n * w + 4 * (n // 2) ** 2 * w))
        for t in range(L):
            add("case1", 6 * n1 * n1 * w + 2 * 3 * n1 * n * C + 2 * 2 * n1 * n * C)
            for s in range(L):
                if s == t:
                    continue
                d = abs(s - t)
                m = 1 << d
                spec = m * m * 6 * n1 * 2 * n * C
                if s > t:  # Case 2: finer source, m^2 phase slabs of n/m rows
                    add(f"case2_d{d}", spec + 2 * 3 * n1 * n * C * m)
                else:      # Case 3: coarser source, m^2 phase outputs of n/m rows
                    add(f"case3_d{d}", spec + 2 * 2 * n1 * n * C * m)
    tot = sum(out.values())
    return {"bytes": out, "total": tot, "share": {k: v / tot for k, v in out.items()}}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1603_03142_gb300 import sgf, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    nest, sigma = W.config3(n, seed=rank)
    # the benchmark density is tapered to zero well inside the domain, so the
    # zero-rim plan (verified on the device every solve) is valid; the general
    # three-field path is timed beside it and reported in config
    # (--solve-only --solve-precision bf16x: the split-BF16 plan alone, for ncu captures of its kernels)
    plan = sgf.Plan(nest, args.solve_precision if args.solve_only else "fp32", zero_rim=not args.general)
    plan_general = sgf.Plan(nest, "fp32") if not (args.general or args.solve_only) else None
    # the autotuner picks each pass's kernel schedule (same arithmetic; results agree to rounding),
    # unless --schedule fixes it
    if args.schedule == "auto":
        tune = plan.autotune(reps=5)
        if plan_general is not None:
            plan_general.autotune(reps=3)
    else:
        parts = [int(x) for x in args.schedule.split(",")]
        col, inv = parts[0], parts[1]
        plan.set_schedule(col, inv, 0, 0, 0, parts[2] if len(parts) > 2 else 0)
        if plan_general is not None:
            plan_general.set_schedule(0, inv)
        tune = {"chosen": plan.schedule(), "ms": None}
    st = plan.stats()
    # rotating input/output sets so nothing carries over in L2 between steps
    sets = max(2, -(-4 * L2_BYTES // (3 * n * n * 4)))
    base = torch.from_numpy(sigma[0].astype(np.float32)).to(dev)
    sig = [base.roll(shifts=k, dims=1).contiguous() for k in range(sets)]
    fx = [torch.empty_like(base) for _ in range(sets)]
    fy = [torch.empty_like(base) for _ in range(sets)]
    stream = torch.cuda.current_stream(dev)

    def timed(p, steps, clocks=None):
        def step(k):
            if p.potential:
                p.solve_potential_ptrs([sig[k % sets].data_ptr()], [fx[k % sets].data_ptr()], stream)
            else:
                p.solve_ptrs([sig[k % sets].data_ptr()], [fx[k % sets].data_ptr()], [fy[k % sets].data_ptr()], stream)
        for k in range(args.warmup):
            step(k)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        p.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev0.record(stream)
        for k in range(steps):
            step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        p.profile(False)
        p.check()  # raises if the device saw a broken zero-rim guarantee
        ms = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, p.profile_read()

    if world > 1:
        import torch.distributed as dist
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        ms, prof = timed(plan, args.steps)
    ms_step = ms / args.steps
    cells = float(n * n)
    value = world * cells * args.steps / (ms / 1e3)
    if args.solve_only:  # the one plan and its timed solves (small device footprint, for ncu captures)
        if rank == 0:
            print(json.dumps({"mode": "solve-only", "n": n, "ms_per_step": ms_step, "cells_per_s": value,
                              "schedule": plan.schedule(),
                              "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in prof["kernels"].items()
                                            if v["launches"]},
                              "device_bytes": torch.cuda.max_memory_allocated(dev) + st["workspace_bytes"] +
                              st["spectra_bytes"]}), flush=True)
        return
    general = None
    if plan_general is not None:
        gms, gprof = timed(plan_general, args.steps)
        general = {"cells_per_s": world * cells * args.steps / (gms / 1e3), "ms_per_step": gms / args.steps,
                   "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in gprof["kernels"].items()
                                 if v["launches"]},
                   "algorithmic_bytes_per_solve": plan_general.stats()["algorithmic_bytes"]}

    bf16x = None
    if not args.no_bf16x:
        # the split-BF16 tensor-core path side by side: same workload, same launch shape
        plan_bf = sgf.Plan(nest, "bf16x", zero_rim=not args.general)
        plan_bf.autotune(reps=3)
        bms, bprof = timed(plan_bf, args.steps)
        ref_x, ref_y = torch.empty_like(base), torch.empty_like(base)
        plan.solve_ptrs([sig[0].data_ptr()], [ref_x.data_ptr()], [ref_y.data_ptr()], stream)
        plan_bf.solve_ptrs([sig[0].data_ptr()], [fx[0].data_ptr()], [fy[0].data_ptr()], stream)
        torch.cuda.synchronize()
        plan_bf.check()
        scale = max(ref_x.abs().max().item(), ref_y.abs().max().item())
        rel = max((fx[0] - ref_x).abs().max().item(), (fy[0] - ref_y).abs().max().item()) / scale
        bf16x = {"cells_per_s": world * cells * args.steps / (bms / 1e3), "ms_per_step": bms / args.steps,
                 "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in bprof["kernels"].items()
                               if v["launches"]},
                 "rel_linf_vs_fp32": rel}
        plan_bf.close()

    potential = None
    if not args.no_potential:
        # the potential (kernel -1/r, one output) on the same density: its zero-rim
        # plan (one merged real table over sigma alone), like the forces
        plan_phi = sgf.Plan(nest, "fp32", potential=True, zero_rim=not args.general)
        plan_phi.autotune(reps=3)
        pms, pprof = timed(plan_phi, args.steps)
        pst = plan_phi.stats()
        pk = {k: v["ms"] / max(1, v["launches"]) for k, v in pprof["kernels"].items() if v["launches"]}
        # column pass: the forward fields in (1 zero-rim, 3 general), the quarter-stored tables
        # (1 merged, 3), one component out
        N1 = n + 1
        nfp = 3 if args.general else 1
        col_bytes = nfp * N1 * n * 8 + nfp * N1 * N1 * 4 + N1 * n * 8
        potential = {"cells_per_s": world * cells * args.steps / (pms / 1e3), "ms_per_step": pms / args.steps,
                     "schedule": plan_phi.schedule(), "kernel_ms": pk,
                     "algorithmic_bytes_per_solve": pst["algorithmic_bytes"],
                     "solve_gbs": pst["algorithmic_bytes"] / (pms / args.steps / 1e3) / 1e9,
                     "col_roofline": {"achieved_gbs": col_bytes / (pk["col"] / 1e3) / 1e9,
                                      "frac": col_bytes / (pk["col"] / 1e3) / 1e9 / peaks()[0],
                                      "algorithmic_bytes_per_launch": col_bytes}}
        plan_phi.close()

    forest = None
    if not args.no_forest:
        forest = time_forest(args, world, dev, stream)

    # e2e: host buffers through the C ABI, copies inside the timed region.  The
    # pipelined call (sgf_solve_host_many) over a ring of page-locked sets:
    # every step copies its density in and its forces out, overlapping the
    # neighbouring steps' transforms.  The one-call-per-step figure
    # (sgf_solve_host, forces written in place over the link) rides along.
    ring = 3
    pin_s = [torch.from_numpy(W.config3(n, seed=7 + k)[1][0].astype(np.float32)).pin_memory() if k else
             torch.from_numpy(sigma[0].astype(np.float32)).pin_memory() for k in range(ring)]
    pin_x = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(ring)]
    pin_y = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(ring)]
    e2e_steps = max(6, args.steps)
    sel = [k % ring for k in range(e2e_steps)]
    sp = [pin_s[k].data_ptr() for k in sel]
    xp = [pin_x[k].data_ptr() for k in sel]
    yp = [pin_y[k].data_ptr() for k in sel]
    plan.solve_host_many_ptrs(ring, sp[:ring], xp[:ring], yp[:ring], stream)  # staging allocated, warm
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    plan.solve_host_many_ptrs(e2e_steps, sp, xp, yp, stream)
    e2e_s = time.perf_counter() - t0
    for _ in range(2):
        plan.solve_host_ptrs([pin_s[0].data_ptr()], [pin_x[0].data_ptr()], [pin_y[0].data_ptr()], stream)
    t1 = time.perf_counter()
    for k in sel:
        plan.solve_host_ptrs([pin_s[k].data_ptr()], [pin_x[k].data_ptr()], [pin_y[k].data_ptr()], stream)
    serial_s = time.perf_counter() - t1
    # the CPU-GPU link alone: one device-to-host copy of a step's forces and one
    # host-to-device copy of its density, each timed by itself and both at once
    link_s = torch.cuda.Stream(dev)
    dfx = torch.empty((2, n, n), dtype=torch.float32, device=dev)
    hfx = torch.empty((2, n, n), dtype=torch.float32).pin_memory()
    dsg = torch.empty((n, n), dtype=torch.float32, device=dev)

    def link_time(d2h, h2d, reps=5):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for r in range(reps + 1):
            if r == 1:
                ev[0].record(stream)
            if h2d:
                link_s.wait_stream(stream)  # both copies start together
                with torch.cuda.stream(link_s):
                    dsg.copy_(pin_s[0], non_blocking=True)
            if d2h:
                with torch.cuda.stream(stream):
                    hfx.copy_(dfx, non_blocking=True)
            if h2d:
                stream.wait_stream(link_s)
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3 / reps

    t_d2h, t_h2d, t_both = link_time(True, False), link_time(False, True), link_time(True, True)
    if world > 1:
        t = torch.tensor([e2e_s, serial_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s, serial_s = (float(v) for v in t.tolist())
    e2e = {"value": world * cells * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": n * n * 4, "d2h_bytes_per_step": 2 * n * n * 4,
           "steps": e2e_steps,
           "transfer": "sgf_solve_host_many over a ring of 3 page-locked sets: each step's sigma copied in "
                       "and Fx, Fy copied out on two copy streams, overlapping the neighbouring steps' solves",
           "link": {"d2h_gbs": 2 * n * n * 4 / t_d2h / 1e9, "h2d_gbs": n * n * 4 / t_h2d / 1e9,
                    "both_ms": t_both * 1e3,
                    "bound": world * cells / t_both, "frac": (cells * e2e_steps / e2e_s) / (cells / t_both),
                    "what": "a step's copies alone (CUDA events): 128 MiB out and 64 MiB in at once; bound = "
                            "cells per step over that time"},
           "one_call_per_step": {"value": world * cells * e2e_steps / serial_s,
                                 "call": "sgf_solve_host (sigma copied in, Fx, Fy written in place to "
                                         "page-locked host memory by the inverse row pass; waits per step)"}}

    # the batched (256 nests) and serving (Poisson mix) workloads, shortened, on the same GPU
    # (after the end-to-end run: their servers hold most of the device and much page-locked memory)
    batched = serving_runs = None
    if world == 1 and not args.no_nest_workloads:
        import copy
        ba = copy.copy(args)
        ba.steps, ba.warmup = 3, 2
        batched = run_batched(ba, world, rank, local)
        sa = copy.copy(args)
        sa.warmup = 1
        serving_runs = run_serving(sa, world, rank, local, streams=[(args.rate, 15.0), (0.0, 10.0)])
        # every shape of the mix served, none rejected: the shapes over the cap regenerate most of
        # their spectra at every solve (seconds each), so this stream runs at a low rate
        serving_all = run_serving(sa, world, rank, local, streams=[(4.0, 4.0)], stream_large=True)
        if serving_runs is not None and serving_all is not None:
            serving_runs["all_shapes_stream"] = serving_all
        import gc
        gc.collect()  # the servers' plans, spectra and page-locked request buffers
        torch.cuda.empty_cache()

    if rank != 0:
        return
    # roofline of the dominant kernel
    peak, peak_kind = peaks()
    kern = prof["kernels"]
    dom = max(kern, key=lambda k: kern[k]["ms"])
    C = 8  # complex64 bytes
    N1 = n + 1
    nf, nt = (3, 6) if args.general else (1, 2)  # forward fields and spectra tables of the timed path
    algo = {"row_fwd": n * n * 4 + nf * N1 * n * C,
            "col": nf * N1 * n * C + nt * N1 * N1 * 4 + 2 * N1 * n * C,
            "row_inv": 2 * N1 * n * C + 2 * n * n * 4,
            "restrict": 0}
    avg_ms = kern[dom]["ms"] / max(1, kern[dom]["launches"])
    achieved = algo[dom] / (avg_ms / 1e3) / 1e9
    total_ms = sum(v["ms"] for v in kern.values())
    traffic = recorded_traffic(dom)
    pipe = recorded_ncu(dom, "fp32_pipe_per_launch")
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample_rate(n, seconds=args.ref_seconds)
        cpu.pop("seconds", None)
        cpu.pop("targets", None)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"uniform-{n}x{n}-lognormal-taper", "n": n, "levels": 1,
                   "precision": "fp32", "parallelism": f"replicas{world}",
                   "path": "general-3-field" if args.general else "zero-rim-merged (verified per solve)",
                   "schedule": tune["chosen"], "autotune_ms": tune["ms"],
                   "general_path": general,
                   "bf16x_path": bf16x,
                   "potential_path": potential,
                   "forest_path": forest,
                   "batched_path": None if batched is None else {
                       "workload": batched["config"]["workload"], "cells_per_s": batched["value"],
                       "ms_per_batch": batched["ms_per_step"], **{k: batched["config"][k] for k in (
                           "nests", "cells_per_batch", "shapes", "kernel_groups", "launches_per_batch", "plan_s",
                           "spectra_gib", "algorithmic_bytes_per_batch", "roofline", "bytes_by_pair")}},
                   "serving_path": serving_runs,
                   "l2": f"{sets} rotating input/output sets ({sets * 3 * n * n * 4 / 2**20:.0f} MiB) > 129 MiB L2",
                   "plan_ms": st["plan_ms"], "spectra_mib": st["spectra_bytes"] / 2**20,
                   "algorithmic_bytes_per_solve": st["algorithmic_bytes"],
                   "solve_gbs": st["algorithmic_bytes"] / (ms_step / 1e3) / 1e9},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": algo[dom],
                     "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in kern.items() if v["launches"]},
                     "kernel_share": {k: v["ms"] / total_ms for k, v in kern.items() if v["launches"]},
                     # the FP32 roof beside the HBM one: the same kernel's FMA-pipe and issue activity
                     # from the committed ncu capture (null once its sources change)
                     "fp32_pipe": None if pipe is None else {
                         "fma_pipe_active": pipe["fma_pipe_active_pct"] / 100.0,
                         "issue_active": pipe["issue_active_pct"] / 100.0, "source": "ncu, profiles/traffic.json"}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * st["launches_per_solve"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_nest_solves(args, world, rank, local):
    """--solve-only --nest-levels L: one general FP32 nest plan (the concentric
    nest of the batched workload, n x n cells a level) and its timed solves on
    two rotating sets of device buffers; prints a short line (a small device
    footprint, for ncu captures of the nest kernels)."""
    import numpy as np
    import torch
    from paper_1603_03142_gb300 import sgf, workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.Generator(np.random.PCG64(args.seed + rank))
    nest, sigma = W.random_nest_problem(rng, args.n, args.nest_levels)
    plan = sgf.Plan(nest, "fp32")
    if args.schedule == "auto":
        plan.autotune(reps=3)
    else:
        parts = [int(x) for x in args.schedule.split(",")]
        plan.set_schedule(parts[0], parts[1], 0, 0, 0, parts[2] if len(parts) > 2 else 0)
    sig = [[torch.from_numpy(a.astype(np.float32)).to(dev).roll(shifts=k, dims=1).contiguous() for a in sigma]
           for k in range(2)]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    stream = torch.cuda.current_stream(dev)

    def step(k):
        q = k % 2
        plan.solve_ptrs([a.data_ptr() for a in sig[q]], [a.data_ptr() for a in fx[q]],
                        [a.data_ptr() for a in fy[q]], stream)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    plan.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    plan.profile(False)
    plan.check()
    prof = plan.profile_read()
    ms = ev0.elapsed_time(ev1) / args.steps
    if rank == 0:
        print(json.dumps({"mode": "solve-only", "n": args.n, "levels": args.nest_levels, "ms_per_step": ms,
                          "cells_per_s": args.nest_levels * args.n * args.n / (ms / 1e3),
                          "schedule": plan.schedule(),
                          "kernel_ms": {k: v["ms"] / max(1, v["launches"]) for k, v in prof["kernels"].items()
                                        if v["launches"]},
                          "device_bytes": torch.cuda.max_memory_allocated(dev) + plan.stats()["workspace_bytes"] +
                          plan.stats()["spectra_bytes"]}), flush=True)


def run_batched(args, world, rank, local):
    """Batched workload: independent concentric nests of uneven N and level
    count solved as one fused batch (sgf_batch_*).  value = all cells of all
    levels of all nests / device time per batch solve.  Nests shard across ranks
    by cost (replicas: no data-path collective)."""
    import numpy as np
    import torch
    from paper_1603_03142_gb300 import replicas, sgf, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    probs = W.config4(count=args.nests, seed=0)
    costs = [replicas.nest_cost(nest.n, nest.levels) for nest, _ in probs]
    mine = replicas.shard_by_cost(costs, rank, world)
    t0 = time.perf_counter()
    base, plans = {}, []
    for k in mine:
        nest = probs[k][0]
        key = nest.key()
        if key not in base:
            base[key] = sgf.Plan(nest, "fp32")
            base[key].autotune(reps=2)  # shared plans start from this schedule; a batch group from its first plan's
            plans.append(base[key])
        else:
            plans.append(base[key].share())
    plan_s = time.perf_counter() - t0
    sig = [[torch.from_numpy(a.astype(np.float32)).to(dev) for a in probs[k][1]] for k in mine]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    batch = sgf.Batch(plans)
    info = batch.info()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        batch.solve(sig, fx, fy, stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            batch.solve(sig, fx, fy, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cells = sum(probs[k][0].levels * probs[k][0].n ** 2 for k in range(len(probs)))
    spectra_gib = sum(p.stats()["spectra_bytes"] for p in base.values()) / 2**30
    algo = sum(plans[i].stats()["algorithmic_bytes"] for i in range(len(plans)))
    pairs = nest_pair_bytes([probs[k][0] for k in mine])
    batch.close()
    for p in plans:
        p.close()
    if rank != 0:
        return None
    shapes = sorted({(p.n, p.levels) for p in base.values()})
    peak = peaks()[0]
    line = {"metric": METRIC, "value": cells * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched-{args.nests}-nests-N128-1024-L1-4", "nests": args.nests,
                       "cells_per_batch": cells, "parallelism": f"replicas{world}", "shapes": len(shapes),
                       "kernel_groups": info["groups"], "launches_per_batch": info["launches_per_solve"],
                       "graph": True, "plan_s": plan_s,
                       "spectra_gib": spectra_gib,
                       "algorithmic_bytes_per_batch": algo,
                       "roofline": {"bound": "hbm", "achieved": algo / (ms / args.steps / 1e3) / 1e9, "peak": peak,
                                    "unit": "GB/s", "frac": algo / (ms / args.steps / 1e3) / 1e9 / peak,
                                    "scope": "whole batch solve (all passes), rank 0's nests"},
                       "bytes_by_pair": pairs},
            "gpu_launches": args.steps * info["launches_per_solve"], "clocks": clk.summary()}
    return line


def run_serving(args, world, rank, local, streams=None, stream_large=False):
    """Serving workload: an open-loop Poisson stream of force requests with host
    buffers, served by the request loop (sgf_server_*): continuous admission by
    HBM footprint onto concurrent streams, spectra resident per shape.  Every
    shape is warmed once (spectra built) before the timed stream.  value = cells
    of the completed requests / span from the first arrival to the last
    completion; latency percentiles over the timed stream.  Each rank serves its
    own stream (replicas: seed + rank).

    stream_large: serve the shapes over the per-shape cap with plans over a
    spectra budget (SGF_SERVER_STREAM) instead of rejecting them.
    streams: None (one stream at args.rate for args.seconds; returns its line)
    or a list of (rate, seconds) run one after the other on the same warmed
    server (returns one summary per stream); a rate of 0 means 85 % of the
    accepted load the previous stream's device sustained."""
    import numpy as np
    import torch
    from paper_1603_03142_gb300 import serving, sgf

    torch.cuda.set_device(local)
    sizes = tuple(int(x) for x in args.sizes.split(","))
    lv = tuple(int(x) for x in args.levels.split(","))
    precs = tuple(args.precisions.split(","))
    plan_streams = streams if streams is not None else [(args.rate, args.seconds)]
    # every shape the mix can draw is warmed, whatever the first stream happens to contain
    shapes = sorted({(n, L, p) for n in sizes for L in range(lv[0], lv[-1] + 1) for p in precs})
    t0 = time.perf_counter()
    pools = serving.make_pools(shapes, seed=args.seed)
    pool_s = time.perf_counter() - t0
    budget = int(args.budget_gb * 2 ** 30)
    srv = sgf.Server(hbm_budget=budget, max_inflight=args.inflight, max_shape_bytes=int(args.max_shape_gb * 2 ** 30),
                     stream_large=stream_large)
    # warm-up: one request per shape (builds and keeps its spectra), then a short stream
    t0 = time.perf_counter()
    warm = [serving.Arrival(0.0, n, L, p, 0) for (n, L, p) in shapes]
    wrec, _ = serving.run_stream(srv, warm, pools, id_base=10 ** 8)
    first = serving.poisson_arrivals(plan_streams[0][0], plan_streams[0][1], args.seed + rank, sizes,
                                     (lv[0], lv[-1]), precs)
    for k in range(max(0, args.warmup - 1)):
        serving.run_stream(srv, first[: max(1, len(first) // 20)], pools, id_base=10 ** 8 + (k + 1) * 10 ** 6)
    warm_s = time.perf_counter() - t0
    accepted = sorted({(r.n, r.levels) for r in wrec if r.status == sgf.SGF_OK})
    rejected_shapes = sorted({(r.n, r.levels) for r in wrec if r.status != sgf.SGF_OK})
    results = []
    prev = None
    for si, (rate, seconds) in enumerate(plan_streams):
        if rate <= 0:  # 85 % of the accepted load the device sustained in the previous stream
            acc_frac = max(1e-3, 1.0 - prev["load"]["rejected"] / max(1, prev["requests"]))
            rate = 0.85 * prev["load"]["achieved_rps"] / acc_frac
        arr = serving.poisson_arrivals(rate, seconds, args.seed + rank + 1000 * si, sizes, (lv[0], lv[-1]), precs)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        with ClockSampler(local) as clk:
            recs, _ = serving.run_stream(srv, arr, pools, id_base=10 ** 9 * (si + 1))
        summ = serving.summarize(recs, seconds)
        launches, h2d, d2h = 0, 0, 0
        for r in recs:
            if r.status == sgf.SGF_OK:
                launches += (r.levels - 1) + 3 + (1 if r.levels > 1 else 0)
                h2d += r.levels * r.n * r.n * 4
                d2h += 2 * r.levels * r.n * r.n * 4
        done = max(1, summ.get("completed", 0))
        value = summ.get("cells_per_s", 0.0)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([value], device=torch.device("cuda", local), dtype=torch.float64)
            dist.all_reduce(t)
            value = float(t.item())
        res = {"offered_rps": rate, "seconds": seconds, "requests": len(recs), "cells_per_s": value,
               "latency_ms": {k: summ.get(k) for k in ("p50_ms", "p90_ms", "p99_ms", "max_ms", "mean_ms")},
               "load": {"offered_rps": summ.get("offered_rps"), "achieved_rps": summ.get("achieved_rps"),
                        "offered_cells_per_s": summ.get("offered_cells_per_s"), "completed": summ.get("completed"),
                        "rejected": summ.get("rejected"), "failed": summ.get("failed")},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d / done,
                       "d2h_bytes_per_step": d2h / done},
               "gpu_launches": launches, "clocks": clk.summary(), "mean_ms": summ.get("mean_ms")}
        results.append(res)
        prev = res
    st = srv.stats()
    srv.close()
    if rank != 0:
        return None
    common = {"shapes": len(shapes), "shapes_served": accepted, "shapes_rejected": rejected_shapes,
              "shapes_over_cap_streamed": bool(stream_large),
              "hbm_budget_gib": args.budget_gb, "max_shape_gib": args.max_shape_gb,
              "max_inflight": args.inflight, "parallelism": f"replicas{world}", "pool_s": pool_s,
              "warm_s": warm_s, "inputs": "pinned host buffers, copies inside the latency",
              "server": {k: st[k] for k in ("inflight_peak", "slots", "shapes_resident", "shapes_built",
                                            "slots_evicted", "bytes_peak")}}
    if streams is not None:
        return {"streams": results, **common}
    r = results[0]
    line = {"metric": METRIC, "value": r["cells_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": r["load"]["completed"] or 0, "warmup": args.warmup, "ms_per_step": r["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving-poisson-{args.rate:g}rps-{args.seconds:g}s-N{sizes[0]}-{sizes[-1]}"
                                   f"-L{lv[0]}-{lv[-1]}-{'+'.join(precs)}",
                       "requests": r["requests"], **common},
            "latency_ms": r["latency_ms"], "load": r["load"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--general", action="store_true", help="time only the general three-field path")
    ap.add_argument("--no-bf16x", action="store_true", help="skip the split-BF16 tensor-core path")
    ap.add_argument("--no-potential", action="store_true", help="skip the potential (SGF_PLAN_POTENTIAL) timing")
    ap.add_argument("--no-forest", action="store_true", help="skip the two-disk forest (Example 3) timing")
    ap.add_argument("--solve-only", action="store_true",
                    help="only the timed solves of the one plan (no other path, no e2e); prints a short line")
    ap.add_argument("--solve-precision", default="fp32", choices=["fp32", "bf16x"],
                    help="with --solve-only: the precision of the one plan")
    ap.add_argument("--nest-levels", type=int, default=0,
                    help="with --solve-only: a general FP32 nest of this many levels (n x n cells each) instead")
    ap.add_argument("--no-nest-workloads", action="store_true",
                    help="uniform: skip the shortened batched and serving runs reported in config")
    ap.add_argument("--forest-n", type=int, default=512, help="cells per side of every patch of the forest")
    ap.add_argument("--schedule", default="auto",
                    help="uniform: 'auto' (autotuner) or 'col_pass,row_inv0[,row_fwd]' to fix the kernel schedule")
    ap.add_argument("--workload", default="uniform", choices=["uniform", "batched", "serving"])
    ap.add_argument("--nests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--seconds", type=float, default=30.0, help="serving: length of the arrival stream")
    ap.add_argument("--sizes", default="256,512,1024,2048", help="serving: n of the requests")
    ap.add_argument("--levels", default="2,5", help="serving: min,max levels of the requests")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: server HBM budget (GiB)")
    ap.add_argument("--inflight", type=int, default=4, help="serving: requests on the device at once")
    ap.add_argument("--max-shape-gb", type=float, default=24.0,
                    help="serving: largest spectra + generator memory of one shape (GiB); larger shapes are rejected")
    ap.add_argument("--precisions", default="fp32,bf16x", help="serving: precisions drawn uniformly per request")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit without work
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        args.ref_seconds = min(args.ref_seconds, max(1.0, 90.0 / (args.steps + args.warmup)))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup()
    if args.workload in ("batched", "serving"):
        line = (run_batched if args.workload == "batched" else run_serving)(args, world, rank, local)
        if line is not None:
            print(json.dumps(line), flush=True)
    elif args.solve_only and args.nest_levels > 0:
        run_nest_solves(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
