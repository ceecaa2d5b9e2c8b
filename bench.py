"""Benchmark of the LBFS time step on GB300.

Default workload: the 4096 x 2048 sessile ferrofluid drop (R = 768, field at 45
degrees, Bo_m = 1.0, chi = 1, Ste = 0.1) in mixed precision (FP32 bulk, FP64
enthalpy accuracy from FP32 pairs, FP64-refined FP32 multigrid potential).  One step
is one full time step of every cell: the potential solve and three Runge-Kutta
stages.  The metric is cell-updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the case (the cases
are independent; there is no collective on the data path) and rank 0 prints one
JSON line with the aggregate over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LBFS Mcell-updates/s"
UNIT = "Mcell-updates/s"
L2_BYTES = 129 * 2 ** 20
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes per cell of one stage launch, averaged over the three stages:
# stage 1 reads W^n, F_s^{n-1}, phi and writes W^1; stages 2 and 3 also read W^n
# cell-locally; stage 3 also writes F_s^n and mu_m.  W is H_e (8 bytes: FP64, or an
# FP32 pair in mixed precision) plus p, m_x, m_y, C in the working precision.
def stage_bytes_per_cell(prec: int) -> float:
    r = 8 if prec == 0 else 4
    w = 8 + 4 * r
    s1 = w + r + r + w
    s2 = w + w + r + r + w
    s3 = w + w + r + r + w + r + r
    return (s1 + s2 + s3) / 3.0


# algorithmic bytes per cell of the potential solve of one step: the step's first
# residual pass (read phi, mu_m; write r), then per refinement cycle the fine level's
# down leg (read mu_m, r; write e; the restriction a quarter of that), its up leg (read
# mu_m, r, e and a quarter cell of coarse correction; write e), the coarser levels (a
# third of the fine level's legs), the correction (read phi and e, write phi) and the
# residual pass again.  phi is 8 bytes (FP64, or an FP32 pair in mixed precision).
def potential_bytes_per_cell(prec: int, cycles: float) -> float:
    r = 8 if prec == 0 else 4
    resid = 8 + r + r
    down = 3 * r + (2 * r) / 4
    up = 4 * r + r / 4
    cycle = (down + up) * 4 / 3 + (8 + r + 8) + resid
    return resid + cycles * cycle


def workloads():
    from paper_2511_10257_gb300 import inputs as I
    return {
        "huge": ("4096x2048 sessile ferrofluid drop, R=768, field 45 deg, Bo_m=1.0, chi=1, Ste=0.1",
                 I.config_huge()),
        "large": ("1024x512 sessile ferrofluid drop, R=192, horizontal field, Bo_m=1.5, chi=2, Ste=0.05",
                  I.config_large()),
        "medium": ("512x256 sessile ferrofluid drop, R=96, vertical field, Bo_m=1.0, chi=1, Ste=0.1",
                   I.config_medium()),
        "small": ("128x64 sessile ferrofluid drop, R=24, vertical field, Bo_m=0.5, chi=1, Ste=0.1",
                  I.config_small()),
        "batch": ("64-case seeded sweep (SplitMix64 seed 0): grids 128x64..512x256, R=0.375 ny, "
                  "field angle 0-90 deg, Bo_m 0-2, Ste 0.05-0.2, chi=1", I.sweep_cases(64, 0)),
    }


def sample_case(case: dict, factor: int) -> dict:
    """the same physics on a grid coarser by `factor` (radius scaled with it)"""
    d = dict(case)
    d["nx"] //= factor
    d["ny"] //= factor
    d["radius"] = case["radius"] / factor
    return d


def reduce_over_ranks(elapsed_s: float, units: float, world: int):
    """max elapsed time and total units over ranks (no-op on one rank)"""
    if world <= 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64)
    u = torch.tensor([units], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t, u = t.cuda(), u.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def stage_source_hash() -> str:
    """hash of the stage kernel's code (comments and blank lines left out): profiled
    counters apply only to this version"""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("lbfs_stage.cu", "lbfs_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2511_10257_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [re.sub(r"//.*", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def profiled(tile_name: str, grid: str, key: str):
    """a per-launch counter of the stage kernel from the committed ncu summary of this
    kernel version and grid, for the tile shape the autotuner kept (None when the
    kernel changed since the capture or the shape was not captured):
    dram_bytes_per_launch_avg or warp_inst_per_launch"""
    path = os.path.join(ROOT, "profiles", "stage_kernel_4096x2048.md")
    try:
        common, tiles, cur = {}, {}, None
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                k, v = k.strip(), v.strip().strip("`")
                if k == "tile":
                    cur = tiles.setdefault(v, {})
                else:
                    (common if cur is None else cur)[k] = v
        if (common.get("source_sha256") == stage_source_hash() and common.get("grid") == grid
                and tile_name in tiles):
            return float(tiles[tile_name][key])
    except Exception:
        return None
    return None


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region"""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)   # the sample that falls due at the end of the timed region
        self.proc.terminate()
        self.proc.wait()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.out.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(case: dict, steps: int, warmup: int, threads: int):
    """FP64 CPU oracle, as it stands, on `case`: cell-updates per second"""
    import oracle
    o = oracle.Oracle(case, threads=threads)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return case["nx"] * case["ny"] * steps / dt / 1e6, dt


def oracle_fullgrid_rate(case: dict, threads: int):
    """FP64 CPU oracle, as it stands, on the workload's own grid: one time step (three
    Runge-Kutta stages) from the workload's initial state, with the potential held at its
    far-field start (the oracle's conjugate-gradient potential solve runs on one core and
    would take minutes per step on this grid, so it is left out, which favours the oracle)."""
    import oracle
    o = oracle.Oracle(dict(case, flags=oracle.FLAG_KEEP_POTENTIAL), threads=threads)
    t0 = time.perf_counter()
    o.step(1)
    dt = time.perf_counter() - t0
    return case["nx"] * case["ny"] / dt / 1e6, dt


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    name, work = workloads()[args.workload]
    threads = args.threads if args.threads > 0 else (os.cpu_count() or 1)
    if isinstance(work, list):
        # the sweep: its first cases, each advanced the full step count
        sub = work[:args.ref_cases]
        ncs = sum(c["nx"] * c["ny"] for c in sub)
        t0 = time.perf_counter()
        for c in sub:
            oracle_rate(c, args.steps, args.warmup, threads)
        dt = time.perf_counter() - t0
        value = ncs * args.steps / dt / 1e6
        case = work[0]
        sample_desc = (f"the first {len(sub)} cases of the sweep ({ncs} cells), {args.steps} steps each after "
                       f"{args.warmup} warm-up steps, {threads} OpenMP threads")
    else:
        case = work
        # grids up to 512x256 run whole; larger ones on a grid coarser by sample_factor
        factor = 1 if case["nx"] * case["ny"] <= 512 * 256 else args.sample_factor
        sample = sample_case(case, factor)
        value, dt = oracle_rate(sample, args.steps, args.warmup, threads)
        what = "the workload itself" if factor == 1 else (
            f"the {name} physics on a {sample['nx']}x{sample['ny']} grid (R={sample['radius']:g})")
        sample_desc = (f"{what}, {args.steps} steps after {args.warmup} warm-up steps, {threads} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": name, "grid": f"{case['nx']}x{case['ny']}",
                                        "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "cpu": cpu_model(), "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def potential_compare(device: int, tol: float = 1e-8, chunk: int = 20000, max_iters: int = 2000000) -> dict:
    """The paper's own magnetic solver (explicit pseudo-time magnetic LBFS) against the
    multigrid solve on the 128x64 drop in FP64: time for each to produce the potential
    from the far-field start, the pseudo-time iteration stopped once it is within tol
    (relative L-infinity) of the multigrid result."""
    from paper_2511_10257_gb300 import inputs as I
    from paper_2511_10257_gb300 import lbfs

    case = I.config_small()
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1, device=device)
    s.set_case(0, case)
    s.timing(True)
    st = s.step(1)[0]
    mg_ms = s.timing_read()[lbfs.TIMING_POTENTIAL][0]
    ref = s.field(0, I.PHI)
    s.close()
    mu_max = 1.0 + max(case["chi_l"], case["chi_s"], case["chi_g"])
    dtau = 0.9 / (4.0 * mu_max)   # forward-Euler limit 1/(4 max mu_m)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1, device=device)
    s.set_case(0, case)
    iters, err = 0, float("inf")
    t0 = time.perf_counter()
    while iters < max_iters:
        s.potential_pseudo_time(0, chunk, dtau)
        iters += chunk
        err = float(abs(s.field(0, I.PHI) - ref).max() / abs(ref).max())
        if err <= tol:
            break
    pt_ms = 1e3 * (time.perf_counter() - t0)
    s.close()
    return {"case": "128x64 sessile drop R=24, vertical field, Bo_m=0.5, chi=1 (FP64, far-field start)",
            "multigrid": {"ms": mg_ms, "cycles": st["pot_cycles"], "rel_residual": st["pot_resid"]},
            "pseudo_time_lbfs": {"ms": pt_ms, "iters": iters, "dtau": dtau, "rel_error_vs_multigrid": err,
                                 "tol": tol, "converged": err <= tol}}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2511_10257_gb300 import build as B
    from paper_2511_10257_gb300 import inputs as I
    from paper_2511_10257_gb300 import lbfs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    name, work = workloads()[args.workload]
    cases = work if isinstance(work, list) else [work]
    case = cases[0]
    prec = lbfs.FP64 if args.precision == "fp64" else lbfs.MIXED
    stream = torch.cuda.current_stream()
    solver = lbfs.Solver(precision=prec, max_cases=len(cases), device=local, stream=stream.cuda_stream,
                         torch_alloc=True, tile=max(args.tile, 0), use_graph=True,
                         mg_plain_cycles=args.plain_cycles)
    for k, c in enumerate(cases):
        solver.set_case(k, c)
    ncell = sum(c["nx"] * c["ny"] for c in cases)
    solver.step(1)
    if args.tile >= 0:
        tile, tile_ms = args.tile, []
    else:
        tile, tile_ms = solver.autotune(reps=3)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    solver.step(args.warmup)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    # per-kernel events run eagerly; --graph 1 times graph replay without them
    solver.timing(not args.graph)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    timed_stats = solver.step(args.steps)
    ev1.record(stream)
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    (st_ms, st_n), (pot_ms, pot_n), (fin_ms, fin_n) = solver.timing_read()
    launches = solver.last_launch_count()
    solver.timing(False)
    clk = clocks.stop()
    t_max, units = reduce_over_ranks(elapsed, ncell * args.steps, world)
    value = units / t_max / 1e6

    # end to end through the C ABI with host buffers: upload the case state from
    # pinned host memory, K steps each returning its statistics, download C, F_l, T
    e2e = None
    if not args.no_e2e:
        in_ids = sorted([I.HE, I.P, I.C, I.MX, I.MY, I.FSPREV, I.PHI])
        out_ids = sorted([I.C, I.FL, I.T])
        hosts, outs = [], []
        for k, c in enumerate(cases):
            host = torch.empty((len(in_ids), c["ny"], c["nx"]), dtype=torch.float64, pin_memory=True).numpy()
            solver.fields_into(k, in_ids, host)
            hosts.append(host)
            outs.append(torch.empty((len(out_ids), c["ny"], c["nx"]), dtype=torch.float64,
                                    pin_memory=True).numpy())
        stats_bytes = 88 * len(cases)   # one lbfs_case_stats per case
        # one untimed step records and instantiates the step graph the job replays
        solver.step(1)
        barrier()
        t0 = time.perf_counter()
        for k, host in enumerate(hosts):
            solver.set_fields_packed(k, in_ids, host)
        for _ in range(args.steps):
            solver.step(1)
        for k in range(len(cases)):
            solver.fields_into(k, out_ids, outs[k])
        barrier()
        t_e2e = time.perf_counter() - t0
        t_e2e, units_e2e = reduce_over_ranks(t_e2e, ncell * args.steps, world)
        e2e = {"value": units_e2e / t_e2e / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(len(in_ids) * 8 * ncell / args.steps),
               "d2h_bytes_per_step": int(stats_bytes + len(out_ids) * 8 * ncell / args.steps),
               "job": "upload the state from pinned host memory, step by step with the statistics "
                      "returned each step, download C, F_l and T"}

    # plain FP64 path on the same grid for the mixed-versus-FP64 speed-up
    fp64 = None
    if prec == lbfs.MIXED and args.fp64_steps > 0:
        s64 = lbfs.Solver(precision=lbfs.FP64, max_cases=len(cases), device=local, stream=stream.cuda_stream,
                          torch_alloc=True)
        for k, c in enumerate(cases):
            s64.set_case(k, c)
        s64.step(2)
        barrier()
        # eager launches with per-kernel-class events, so the step splits into stage,
        # potential and step-end time
        s64.timing(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st64 = s64.step(args.fp64_steps)
        b.record(stream)
        barrier()
        t64 = a.elapsed_time(b) / 1e3
        (s_ms, s_n), (p_ms, p_n), (f_ms, f_n) = s64.timing_read()
        s64.timing(False)
        s64.close()
        fp64 = {"value": ncell * args.fp64_steps / t64 / 1e6, "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": 1e3 * t64 / args.fp64_steps,
                "stage_ms_per_launch": s_ms / max(s_n, 1),
                "stage_bytes_per_cell": stage_bytes_per_cell(lbfs.FP64),
                "potential_ms_per_step": p_ms / max(p_n, 1),
                "finalize_ms_per_step": f_ms / max(f_n, 1),
                "pot_resid_max": max(x["pot_resid_max"] for x in st64),
                "pot_cycles_mean": sum(x["pot_cycles_mean"] for x in st64) / len(st64)}

    if rank != 0:
        solver.close()
        return 0
    peak, peak_kind = measured_peak()
    bpc = stage_bytes_per_cell(prec)
    stage_avg_s = st_ms / max(st_n, 1) / 1e3 if st_n else float("nan")
    achieved = ncell * bpc / stage_avg_s / 1e9
    gname = f"{case['nx']}x{case['ny']}"
    traffic = profiled(lbfs.TILE_NAMES[tile], gname, "dram_bytes_per_launch_avg") if len(cases) == 1 else None
    winst = profiled(lbfs.TILE_NAMES[tile], gname, "warp_inst_per_launch") if len(cases) == 1 else None
    # issue roofline: 152 SMs x 4 schedulers issue one warp instruction per clock each
    sm_mhz = clk.get("sm_mhz") or 2070.0
    issue_peak = 152 * 4 * sm_mhz * 1e6
    issue = None
    if winst is not None:
        issue = {"achieved_warp_inst_per_s": winst / stage_avg_s, "peak_warp_inst_per_s": issue_peak,
                 "frac": winst / stage_avg_s / issue_peak,
                 "note": "executed instructions per launch from the committed ncu capture"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "stage_kernel",
                "peak_source": peak_kind, "bytes_per_cell": bpc,
                "launch_ms": stage_avg_s * 1e3, "issue": issue,
                "potential_ms_per_step": pot_ms / max(pot_n, 1),
                "finalize_ms_per_step": fin_ms / max(fin_n, 1)}
    # the potential solve of every timed step, after its last cycle
    potential = {"tol": solver.mg_tol_used(),
                 "resid_max": max(x["pot_resid_max"] for x in timed_stats),
                 "cycles_mean": sum(x["pot_cycles_mean"] for x in timed_stats) / len(timed_stats),
                 "all_converged": all(x["pot_resid_max"] <= solver.mg_tol_used() for x in timed_stats)}
    # the whole step against the same peak: three stage launches plus the potential's
    # passes at the cycle count the timed steps ran
    b_step = 3 * bpc + potential_bytes_per_cell(prec, potential["cycles_mean"])
    roofline["step"] = {"bytes_per_cell": b_step, "achieved": value * 1e6 * b_step / 1e9,
                        "frac": value * 1e6 * b_step / 1e9 / peak, "unit": "GB/s",
                        "potential_bytes_per_cell": b_step - 3 * bpc}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        if len(cases) == 1:
            v, dt = oracle_fullgrid_rate(case, threads)
            cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
                   "sample": f"the workload itself ({case['nx']}x{case['ny']}): one step of three Runge-Kutta "
                             f"stages from its initial state, {dt:.1f} s; the potential is held at its far-field "
                             f"start (the oracle's serial potential solve is left out, which favours the oracle)"}
        else:
            sub = cases[:8]
            ncs = sum(c["nx"] * c["ny"] for c in sub)
            t0 = time.perf_counter()
            for c in sub:
                oracle_rate(c, args.cpu_steps, 0, threads)
            dt = time.perf_counter() - t0
            cpu = {"value": ncs * args.cpu_steps / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "cpu": cpu_model(),
                   "sample": f"the first 8 cases of the sweep ({ncs} cells), {args.cpu_steps} full steps each, "
                             f"{dt:.1f} s"}
    pcmp = None if args.no_potential_compare or world > 1 else potential_compare(local)
    state_bytes = ncell * (8 + 4 * (8 if prec == 0 else 4))
    grid = f"{case['nx']}x{case['ny']}" if len(cases) == 1 else f"{len(cases)} cases, {ncell} cells"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == lbfs.FP64 else "f32+f32x2",
        "data": "synthetic",
        "config": {"workload": name, "grid": grid, "cases": len(cases),
                   "precision": args.precision,
                   "execution": ("timed steps replay the recorded CUDA graph" if args.graph else
                                 "timed steps launch eagerly with per-kernel CUDA events; the e2e job "
                                 "replays the recorded CUDA graph"),
                   "tile": lbfs.TILE_NAMES[tile],
                   "autotune_ms_per_shape": {nm: round(m, 4) for nm, m in zip(lbfs.TILE_NAMES, tile_ms)},
                   "l2": f"inputs larger than L2: per-step working set {3 * state_bytes / 2**20:.0f} MiB "
                         f"(three state sets of {state_bytes / 2**20:.0f} MiB) against 129 MiB of L2, no flush"
                   if 3 * state_bytes > L2_BYTES else "working set fits L2 (no flush)"},
        "roofline": roofline,
        "potential": potential,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "fp64": fp64,
        "potential_solvers": pcmp,
    }
    print(json.dumps(line))
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="huge", choices=["huge", "large", "medium", "small", "batch"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-steps", type=int, default=20, help="oracle steps per case of the batch baseline")
    ap.add_argument("--sample-factor", type=int, default=16,
                    help="reference arm: grids above 512x256 are timed on a grid this much coarser")
    ap.add_argument("--threads", type=int, default=0, help="reference arm: oracle threads (0: all cores)")
    ap.add_argument("--ref-cases", type=int, default=8, help="reference arm, sweep: cases timed")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-potential-compare", action="store_true",
                    help="skip the multigrid versus pseudo-time magnetic LBFS comparison")
    ap.add_argument("--tile", type=int, default=-1, help="stage tile shape id; -1: autotune")
    ap.add_argument("--plain-cycles", action="store_true",
                    help="warm potential cycles as plain launches (for kernel profilers, which cannot follow "
                         "conditional graph nodes)")
    ap.add_argument("--graph", type=int, default=0,
                    help="1: replay recorded CUDA graphs (disables the per-kernel timing)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
