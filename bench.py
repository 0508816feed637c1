#!/usr/bin/env python3
"""Benchmark of the SE k-space path: energy+force evaluations per second.

One step = one whole k-space evaluation (bin, spread, FFT, scale, inverse
FFT, gather; energy, forces and potentials) of the named workload, with the
inputs resident on the GPU.  Between timed steps L2 is flushed by writing a
256 MiB buffer (outside the timed events).  `e2e` times the same evaluation
through the host-buffer entry point (se_energy_force_host: copies in, compute,
copies out).  The accuracy is the relative rms force error against a
high-accuracy FP64 evaluation on the GPU (P = 24, M ~ 4 xi L), which the tests
pin to the direct Ewald sum.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

With torchrun (N > 1) every rank evaluates its own replica of the workload
(the path does not shard a single system); value = all ranks' evaluations per
second of the slowest rank.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "water-L6-M52-P6-fp32comp"
METRIC = "SE k-space energy+force evals/s and ns/atom at stated rms force error vs FP64"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bounded CPU work of the cpu_baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the legs after the headline: accuracy, e2e, at-target, no-graph, "
                         "unsorted variant, autograd, evaluation modes, real space, xi balance "
                         "and cpu_baseline")
    ap.add_argument("--tile", type=int, default=0,
                    help="spreading tile edge (0 = autotune, JSON-cached)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="spread variant (-1 = autotune with the tile; 3 sorted, 4 unsorted)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def system_cost(N, M, P):
    """Work of one system's evaluation: N P^3 for spread and gather, plus
    M^3 log2 M for the transforms."""
    return float(N) * P ** 3 + float(M) ** 3 * math.log2(max(M, 2))


def partition_systems(costs, ws):
    """Systems -> ranks, balanced by cost (largest first onto the least loaded
    rank; ties to the lower rank): every rank computes the same assignment, so
    no exchange is needed.  Returns the sorted system indices of each rank."""
    load = [0.0] * ws
    parts = [[] for _ in range(ws)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(ws), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value, ws, device):
    """The largest value over all ranks (the slowest rank's time)."""
    if ws <= 1:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def workload(name):
    from paper_1712_04718_gb300 import systems
    x, q, w = systems.make(name)
    prec = "fp64" if w["prec"] == "fp64" else "fp32"
    return x, q, w, prec


def dft_split(M):
    """M1 of the factored transforms: the largest divisor of M not above sqrt(M)."""
    best, a = 1, 2
    while a * a <= M:
        if M % a == 0:
            best = a
        a += 1
    return best


def stage_work(w, prec, N, variant, tile=0):
    """Algorithmic work of each own kernel per launch: (kind, amount, kernel).

    spread (variants 3, 4): N P^3 weights; in the sorted pipeline each is one
      native 32-bit shared-memory atomic add ("smem_atomic"), otherwise a
      multiply and an add (2 flops);
    gather: N P^3 grid values, each two FMAs (4 flops);
    single-precision pipeline: the z transforms are direct real DFTs (M^2 rows
      x M inputs x (M/2+1) outputs, 2 FMAs = 4 flops each); the y and x
      transforms are factored complex DFTs, M (M1 + M/M1) complex multiply-adds
      (8 flops) per column of length M; the x pass does two of them and the
      scaling (about 6 flops per mode);
    cuFFT pipeline: scale reads and writes the half spectrum and the G table
      (bytes); bin/scatter: particle bytes."""
    P, M = w["P"], w["M"]
    Mh = M // 2 + 1
    ts = 8 if prec == "fp64" else 4
    nc = M * M * Mh
    fast = variant in (3, 4)
    M1 = dft_split(M)
    cplx = 8.0 * M * (M1 + M // M1) * (M * Mh) if M1 > 1 else 8.0 * M * M * (M * Mh)
    real = 4.0 * M ** 3 * Mh
    work = {
        "spread": (("smem_atomic", float(N) * P ** 3, "k_fspread") if variant == 3 else
                   ("flop", 2.0 * N * P ** 3, "k_fdirect" if variant == 4 else "k_spread")),
        "gather": ("flop", 4.0 * N * P ** 3, "k_fgather" if variant == 3 and
                   tile_gather_selected(N, M, P, tile) else "k_gather"),
        "bin": ("byte", N * (4 * ts + 8), "k_fbin" if variant == 3 else "k_bin"),
        "scatter": ("byte", N * (4 * ts + 4 * ts + 8 + 4), "k_scatter"),
    }
    if fast:
        work["fft_fwd"] = ("flop", real + cplx, "k_slab_fwd")
        work["scale"] = ("flop", 2 * cplx + 6.0 * nc, "k_xpass")
        work["fft_inv"] = ("flop", cplx + real, "k_slab_inv")
    else:
        work["scale"] = ("byte", nc * (4 * ts + 8) + M ** 3 * ts, "k_scale")
    return work


def tile_gather_selected(N, M, P, tile):
    """Whether the single-precision pipeline gathers with its tile kernel
    (k_fgather) rather than k_gather: the library's own rule (dense tiles,
    mean particles per tile x P^3 >= 8 x region, the region with its padded
    rows within 64 KB), restated here only to name the kernel."""
    if not tile:
        return False
    R = tile + P - 1
    RS = P + 15 if P <= 16 else R
    nT = (M + tile - 1) // tile
    ntiles = nT ** 3
    return (R * R * RS * 4 <= 64 * 1024 and ntiles + 8 <= 4096 and
            (N / ntiles) * P ** 3 >= 8.0 * R ** 3)


def kernel_sources_sha():
    """Digest of the single-precision kernel sources (an ncu summary applies
    only to the sources it was taken on)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("se_fast.cuh", "se_fast_launch.cuh", "se_kernels.cuh", "se_dft.cuh",
              "se_internal.h"):
        with open(os.path.join(ROOT, "paper_1712_04718_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cost_model(stages, nstage, N, M, P, variant):
    """The paper's cost model T = c_sp-ga N P^3 + c_fft (M^3/2) log2(M^3/2) +
    c_solve M^3 (Sec. 6.2) with its constants taken from this run's per-stage
    times (direct launches): spread, gather and bin against N P^3, the
    transforms against (M^3/2) log2(M^3/2), the scaling against M^3 (in the
    single-precision pipeline the scaling pass also holds the x transforms).
    The paper's values for one i7-3770 core in FP64 are given beside them."""
    n = max(1, nstage)
    us = {k: v / n * 1e3 for k, v in stages.items()}
    m3 = float(M) ** 3
    fft_units = (m3 / 2.0) * math.log2(m3 / 2.0)
    return {
        "c_spread_gather_s": (us["bin"] + us["scatter"] + us["spread"] + us["gather"]) * 1e-6 /
                             (float(N) * P ** 3),
        "c_fft_s": (us["fft_fwd"] + us["fft_inv"]) * 1e-6 / fft_units,
        "c_solve_s": us["scale"] * 1e-6 / m3,
        "note": "per-stage CUDA events around single launches (launch latency included); "
                "scaling pass includes the x transforms" if variant in (3, 4) else
                "per-stage CUDA events around single launches (launch latency included)",
        "paper_i7_3770_1core_fp64": {"c_spread_gather_s": 5e-9, "c_fft_s": 4.5e-9,
                                     "c_solve_s": 2e-9},
    }


def profiled_traffic(kernel, workload_name):
    """DRAM bytes per launch (read + write) of `kernel` on `workload_name` from
    a committed ncu summary profiles/ncu_<name>_<workload>.md: a line
    `dram_bytes_per_launch.<kernel>: B` (or `dram_bytes_per_launch: B` in the
    summary named for that kernel).  None when no summary holds the kernel or
    the summary was taken on other kernel sources."""
    import glob
    tail = "_%s.md" % workload_name
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "ncu_*" + tail))):
        named = os.path.basename(path)[len("ncu_"):-len(tail)]
        vals = {}
        for line in open(path):
            line = line.strip().lstrip("-* ").strip()
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip().strip("`")] = v.strip().strip("`")
        if vals.get("kernel_sources_sha256") != kernel_sources_sha():
            continue
        v = vals.get("dram_bytes_per_launch.%s" % kernel)
        if v is None and named == kernel:
            v = vals.get("dram_bytes_per_launch")
        if v is None:
            continue
        try:
            return float(v)
        except ValueError:
            return None
    return None


def roofline(kind, amount, kernel, secs, prec, peaks, workload_name):
    """Roofline object of one kernel: achieved rate of its bounding unit over
    that unit's measured peak."""
    from paper_1712_04718_gb300 import se
    if kind == "smem_atomic":
        pk = se.probe_peak("smem_atomic_u32") / 1e9
        achieved = amount / secs / 1e9
        r = {"bound": "alu", "unit": "Gop/s", "peak_source":
             "measured: se_probe_peak shared-memory u32 atomic adds (this run)",
             "fp32_tflops": 2.0 * amount / secs / 1e12}
    elif kind == "flop":
        pk = se.probe_peak("fp64_fma" if prec == "fp64" else "fp32_fma") / 1e12
        achieved = amount / secs / 1e12
        r = {"bound": "alu", "unit": "TFLOP/s", "peak_source":
             "measured: se_probe_peak %s FMA (this run)" % ("FP64" if prec == "fp64" else "FP32")}
    else:
        pk = peaks.get("hbm_gbs", 6800.0)
        achieved = amount / secs / 1e9
        r = {"bound": "hbm", "unit": "GB/s",
             "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}
    r.update({"kernel": kernel, "achieved": achieved, "peak": pk, "frac": achieved / pk,
              "traffic": profiled_traffic(kernel, workload_name),
              "work_per_launch": amount, "launch_us": secs * 1e6})
    return r


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1712_04718_gb300 import se

    if args.workload.startswith("ensemble"):
        return run_ensemble(args, torch, se, ws, rank)
    x, q, w, prec = workload(args.workload)
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
    dt = plan.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    if args.tile or args.variant >= 0:
        plan.set_tuning(max(0, args.variant), args.tile)
    elif prec != "fp64":
        from paper_1712_04718_gb300 import tuning
        tuning.tune_plan(plan, xd, qd)
    variant = plan.params()["spread_variant"]
    tile = plan.params()["tile"]
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush_w = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def flush():
        # write 256 MiB (evicts everything), then read another 256 MiB so that
        # the dirty lines are written back before the timed step starts
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_out)

    def step():
        plan.evaluate(xd, qd, F, phi, Ed)

    for _ in range(max(3, args.warmup)):
        flush()
        step()
    torch.cuda.synchronize()
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(K):
        flush()
        starts[i].record()
        step()
        ends[i].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # stage breakdown: a second pass with per-stage events (direct launches,
    # the graph is not used while timing)
    plan.get_timing(reset=True)
    plan.set_timing(True)
    Ks = min(K, 1000)
    for i in range(Ks):
        flush()
        step()
    torch.cuda.synchronize()
    plan.set_timing(False)
    stages, nstage = plan.get_timing(reset=True)
    total_ms = max_over_ranks(total_ms, ws, "cuda")
    ms_step = total_ms / K
    value = ws * K / (total_ms / 1e3)

    # roofline of the dominant own kernel (average launch duration from events)
    fast = variant in (3, 4)
    work = stage_work(w, prec, N, variant, int(tile or 0))
    per_launch_ms = {k: v / max(1, nstage) for k, v in stages.items()}
    own = [k for k in ("bin", "scatter", "spread", "scale", "gather") if k in work]
    if fast:
        own += ["fft_fwd", "fft_inv"]   # the transforms are own kernels there
    if variant in (3, 4):
        own.remove("scatter")           # no scatter kernel in these pipelines
    if variant == 4:
        own.remove("bin")
    dom = max(own, key=lambda k: per_launch_ms[k])
    kind, amount, kname = work[dom]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    roof = roofline(kind, amount, kname, per_launch_ms[dom] / 1e3, prec, peaks, args.workload)
    roof["measured_unit_peaks"] = {
        "fp32_fma_tflops": se.probe_peak("fp32_fma") / 1e12,
        "fp64_fma_tflops": se.probe_peak("fp64_fma") / 1e12,
        "smem_atomic_u32_gops": se.probe_peak("smem_atomic_u32") / 1e9,
        "smem_atomic_f32_gops": se.probe_peak("smem_atomic_f32") / 1e9,
        "hbm_gbs": peaks.get("hbm_gbs"), "source": "se_probe_peak in this run; HBM from "
        "MEASURED_PEAKS.json"}
    roof["all_kernels"] = {
        work[k][2]: {"us": per_launch_ms[k] * 1e3, "work": work[k][1], "kind": work[k][0]}
        for k in own}

    out = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step,
        "ns_per_atom": ms_step * 1e6 / N, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "L": w["L"], "xi": w["xi"], "M": w["M"],
                   "P": w["P"], "precision": w["prec"], "parallelism": "replicas" if ws > 1 else "single",
                   "spread_variant": variant,
                   "spread_tile": tile if variant != 4 else None,
                   "pipeline": {3: "single-precision, no cuFFT, sorted spread",
                                4: "single-precision, no cuFFT, unsorted spread"}.get(variant, "cuFFT"),
                   "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)"},
        "stages_us_per_eval": {k: v / max(1, nstage) * 1e3 for k, v in stages.items()},
        "stages_note": "per-stage CUDA events, direct launches, %d evaluations (the headline "
                       "replays one CUDA graph per evaluation)" % nstage,
        "fft_us_per_eval": (stages["fft_fwd"] + stages["fft_inv"]) / max(1, nstage) * 1e3,
        "cost_model": cost_model(stages, nstage, N, w["M"], w["P"], variant),
        "roofline": roof,
        "gpu_launches": {3: 6, 4: 5}.get(variant, 5) * K,
        "gpu_launches_note": {
            3: "own kernels per step: bin, spread, slab_fwd, xpass, slab_inv, gather",
            4: "own kernels per step: spread (unsorted), slab_fwd, xpass, slab_inv, gather"}.get(
                variant, "own kernels per step: bin, scatter, spread, scale, gather (+ cuFFT)"),
        "clocks": clk,
    }

    if rank == 0 and not args.no_extras:
        out["accuracy"] = accuracy(se, torch, x, q, w, prec, F)
        out["e2e"] = e2e(se, torch, x, q, w, prec, max(20, min(K, 500)), (variant, tile))
        if args.workload == DEFAULT_WORKLOAD:
            out["at_target"] = at_target(se, torch, x, q, w, prec, K, flush)
        out["no_graph"] = no_graph(se, torch, plan, xd, qd, F, phi, Ed, flush, min(K, 1000))
        if prec != "fp64" and w["M"] <= 128:
            out["unsorted_variant"] = unsorted_variant(se, torch, x, q, w, prec, min(K, 1000), flush)
        out["autograd"] = autograd_timing(se, torch, x, q, w, prec, max(20, min(K, 500)), flush)
        out["modes"] = other_modes(se, torch, x, q, w, prec, min(K, 500), flush, (variant, tile))
        out["real_space"] = real_space(se, torch, x, q, w, prec, min(K, 500), flush, plan)
        if prec != "fp64":
            out["xi_balance"] = xi_balance(se, torch, x, q, w, prec)
        out["cpu_baseline"] = cpu_baseline(x, q, w, args.cpu_seconds)
    plan.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_ensemble(args, torch, se, ws, rank):
    """The batched ensemble: every rank evaluates its share of the systems
    (balanced by cost, partition_systems) through one se_batch; value = evaluations of the whole
    ensemble per second of the slowest rank (strong scaling: the ensemble is
    fixed)."""
    from paper_1712_04718_gb300 import systems, tuning
    w = systems.WORKLOADS[args.workload]
    ens = systems.ensemble(S=w["S"], spacing=w["spacing"])
    parts = partition_systems([system_cost(len(d["q"]), d["M"], w["P"]) for d in ens], ws)
    mine = [ens[i] for i in parts[rank]]
    Ns = [len(d["q"]) for d in mine]
    b = se.Batch(Ns, [d["L"] for d in mine], [d["M"] for d in mine], w["xi"], w["P"])
    xd = torch.tensor(np.concatenate([d["x"] for d in mine]), device="cuda")
    qd = torch.tensor(np.concatenate([d["q"] for d in mine]), device="cuda")
    if args.tile:
        b.set_tile(args.tile)
        tile = args.tile
    else:
        tile, _, _ = tuning.tune_batch(b, xd, qd)
    Ntot = int(sum(Ns))
    F = torch.empty((Ntot, 3), dtype=torch.float32, device="cuda")
    phi = torch.empty((Ntot,), dtype=torch.float32, device="cuda")
    E = torch.empty((len(mine),), dtype=torch.float64, device="cuda")
    flush_w = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def flush():
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_out)

    for _ in range(max(3, args.warmup)):
        flush()
        b.evaluate(xd, qd, F, phi, E)
    torch.cuda.synchronize()
    K = args.steps
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(K):
        flush()
        st[i].record()
        b.evaluate(xd, qd, F, phi, E)
        en[i].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(c) for a, c in zip(st, en))
    total_ms = max_over_ranks(total_ms, ws, "cuda")
    ms_step = total_ms / K
    Nall = sum(len(d["q"]) for d in ens)
    out = {
        "metric": METRIC, "value": K / (total_ms / 1e3), "unit": "ensemble evals/s",
        "n_gpus": ws, "steps": K, "warmup": args.warmup, "ms_per_step": ms_step,
        "ns_per_atom": ms_step * 1e6 / Nall, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "systems": len(ens), "atoms": Nall,
                   "M_range": [min(d["M"] for d in ens), max(d["M"] for d in ens)],
                   "P": w["P"], "xi": w["xi"], "parallelism": "systems sharded over ranks",
                   "spread_tile": tile, "l2": "flushed between steps (untimed)"},
        "gpu_launches": 8 * K, "clocks": clk,
    }
    # per-stage times (direct launches with events between the stages) and the
    # roofline of the dominant stage of spread and gather
    b.set_timing(True)
    for _ in range(20):
        b.evaluate(xd, qd, F, phi, E)
    torch.cuda.synchronize()
    stages, nst = b.get_timing()
    b.set_timing(False)
    us = {k: v / max(1, nst) * 1e3 for k, v in stages.items()}
    out["stages_us_per_eval"] = us
    out["stages_note"] = "per-stage CUDA events, direct launches, %d evaluations" % nst
    P3 = float(w["P"]) ** 3
    if us["spread"] >= us["gather"]:
        pk = se.probe_peak("smem_atomic_u32") / 1e9
        ach = Ntot * P3 / (us["spread"] * 1e-6) / 1e9
        out["roofline"] = {"kernel": "k_bspread", "bound": "alu", "unit": "Gop/s", "achieved": ach,
                           "peak": pk, "frac": ach / pk, "traffic": None,
                           "work": "N P^3 shared-memory atomic adds",
                           "peak_source": "measured: se_probe_peak shared-memory u32 atomics"}
    else:
        pk = se.probe_peak("fp32_fma") / 1e12
        ach = 4.0 * Ntot * P3 / (us["gather"] * 1e-6) / 1e12
        out["roofline"] = {"kernel": "k_bgather_tile / k_bgather", "bound": "alu",
                           "unit": "TFLOP/s", "achieved": ach, "peak": pk, "frac": ach / pk,
                           "traffic": None, "work": "4 N P^3 flops",
                           "peak_source": "measured: se_probe_peak FP32 FMA"}
    if rank == 0 and not args.no_extras:
        # the FP64 oracle on whole systems of the ensemble, in order, until ~5 s
        import oracle
        t0 = time.perf_counter()
        n_done = 0
        k_sys = 0
        for d in ens:
            oracle.se_kspace(np.asarray(d["x"], np.float64), np.asarray(d["q"], np.float64),
                             d["L"], w["xi"], d["M"], w["P"])
            n_done += len(d["q"])
            k_sys += 1
            if time.perf_counter() - t0 > 5.0:
                break
        dt = (time.perf_counter() - t0) * Nall / n_done
        out["cpu_baseline"] = {"value": 1.0 / dt, "unit": "ensemble evals/s",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "the first %d of %d systems (%d atoms), scaled by atoms"
                                         % (k_sys, len(ens), n_done)}
        errs = []
        off = np.concatenate([[0], np.cumsum(Ns)])
        for s in range(0, len(mine), max(1, len(mine) // 4)):
            d = mine[s]
            _, Fref, _ = reference_forces(se, torch, d["x"], d["q"], dict(L=d["L"], xi=w["xi"]))
            errs.append(rel_rms(F[off[s]:off[s + 1]].double().cpu().numpy(), Fref))
        out["accuracy"] = {"rel_rms_force_err_max_sampled": max(errs),
                           "target": w["target_rel_force_err"],
                           "target_met": max(errs) <= w["target_rel_force_err"],
                           "systems_sampled": len(errs)}
        hx = torch.empty_like(xd, device="cpu").pin_memory()
        hq = torch.empty_like(qd, device="cpu").pin_memory()
        hF = torch.empty_like(F, device="cpu").pin_memory()
        hE = torch.empty_like(E, device="cpu").pin_memory()
        hx.copy_(xd)
        hq.copy_(qd)
        k2 = max(10, min(K, 200))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            xd.copy_(hx, non_blocking=True)
            qd.copy_(hq, non_blocking=True)
            b.evaluate(xd, qd, F, phi, E)
            hF.copy_(F, non_blocking=True)
            hE.copy_(E, non_blocking=True)
            torch.cuda.synchronize()
        t1 = time.perf_counter()
        out["e2e"] = {"value": k2 / (t1 - t0), "unit": "ensemble evals/s", "steps": k2,
                      "h2d_bytes_per_step": hx.numel() * 4 + hq.numel() * 4,
                      "d2h_bytes_per_step": hF.numel() * 4 + hE.numel() * 8}
    b.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def reference_forces(se, torch, x, q, w):
    """High-accuracy FP64 SE on the GPU: P = 24, M = 2 ceil(6.2 xi L / pi)
    (Fourier truncation e^-(pi M / 2 xi L)^2 below 1e-16); for workloads whose
    stated error is below 1e-6, P = 32 and a grid at least 16 finer than the
    workload's."""
    M = 2 * math.ceil(6.2 * w["xi"] * w["L"] / math.pi)
    P = 24
    if w.get("target_rel_force_err", 1.0) < 1e-6:
        M, P = max(M, w["M"] + 16), 32
    plan = se.Plan(len(q), w["L"], w["xi"], M, P, precision="fp64")
    E, F, _ = plan.energy_force(torch.tensor(np.asarray(x, np.float64), device="cuda"),
                                torch.tensor(np.asarray(q, np.float64), device="cuda"))
    plan.close()
    return E, F.cpu().numpy(), M


def rel_rms(a, b):
    return float(math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def accuracy(se, torch, x, q, w, prec, F):
    Eref, Fref, Mref = reference_forces(se, torch, x, q, w)
    err = rel_rms(F.double().cpu().numpy(), Fref)
    return {"rel_rms_force_err": err, "target": w["target_rel_force_err"],
            "target_met": err <= w["target_rel_force_err"],
            "reference": "FP64 SE on the GPU, P=%d, M=%d" % (
                32 if w["target_rel_force_err"] < 1e-6 else 24, Mref)}


def at_target(se, torch, x, q, w, prec, K, flush):
    """Same workload at the smallest even P that meets the stated force error."""
    N = len(q)
    Eref, Fref, _ = reference_forces(se, torch, x, q, w)
    for P in (8, 10, 12):
        plan = se.Plan(N, w["L"], w["xi"], w["M"], P, precision=prec)
        dt = plan.dtype
        xd = torch.tensor(x, dtype=dt, device="cuda")
        qd = torch.tensor(q, dtype=dt, device="cuda")
        if prec != "fp64":
            from paper_1712_04718_gb300 import tuning
            tuning.tune_plan(plan, xd, qd)
        F = torch.empty((N, 3), dtype=dt, device="cuda")
        phi = torch.empty((N,), dtype=dt, device="cuda")
        for _ in range(10):
            plan.evaluate(xd, qd, F, phi)
        torch.cuda.synchronize()
        err = rel_rms(F.double().cpu().numpy(), Fref)
        if err > w["target_rel_force_err"]:
            plan.close()
            continue
        k = max(50, min(K, 2000))
        st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for i in range(k):
            flush()
            st[i].record()
            plan.evaluate(xd, qd, F, phi)
            en[i].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / k
        variant = plan.params()["spread_variant"]
        plan.close()
        return {"P": P, "spread_variant": variant,
                "value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms,
                "ns_per_atom": ms * 1e6 / N, "rel_rms_force_err": err, "steps": k}
    return None


def autograd_timing(se, torch, x, q, w, prec, K, flush):
    """The differentiable energy (autograd.se_energy): forward alone (spread
    and scaling, energy from the grid) and forward + backward (the adjoint
    gather: dE/dx, dE/dq), each step launched from Python through
    torch.autograd, timed with CUDA events around the step."""
    from paper_1712_04718_gb300.autograd import se_energy
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
    dt = plan.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    xg = xd.clone().requires_grad_(True)
    qg = qd.clone().requires_grad_(True)

    def fwd():
        with torch.no_grad():
            return se_energy(xd, qd, plan)

    def fwd_bwd():
        xg.grad = None
        qg.grad = None
        se_energy(xg, qg, plan).backward()

    res = {}
    for name, fn in (("forward", fwd), ("forward_backward", fwd_bwd)):
        for _ in range(5):
            fn()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            flush()
            st[i].record()
            fn()
            en[i].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / K
        res[name] = {"value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": K}
    plan.close()
    return res


def unsorted_variant(se, torch, x, q, w, prec, K, flush):
    """The same evaluation with spread variant 4 (no sort: global float
    reductions straight into the grid) instead of the shared-memory tiles."""
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec, spread_variant=4)
    dt = plan.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    for _ in range(10):
        plan.evaluate(xd, qd, F, phi)
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for i in range(K):
        flush()
        st[i].record()
        plan.evaluate(xd, qd, F, phi)
        en[i].record()
    torch.cuda.synchronize()
    plan.close()
    ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / K
    return {"spread_variant": 4, "value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms,
            "steps": K}


def other_modes(se, torch, x, q, w, prec, K, flush, cfg):
    """The workload in the evaluation modes beside the headline's: forces by
    ik differentiation (the cuFFT pipeline with three more inverse FFTs and a
    four-grid gather), potential only (the gather without force sums) and
    energy only (no gather).  Same timing as the headline."""
    N = len(q)
    _, Fref, _ = reference_forces(se, torch, x, q, w)
    out = {}
    for mode in ("ik_forces", "potential_only", "energy_only"):
        plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec,
                       force_mode="ik" if mode == "ik_forces" else "analytic")
        if prec != "fp64":
            plan.set_tuning(*cfg)
        dt = plan.dtype
        xd = torch.tensor(x, dtype=dt, device="cuda")
        qd = torch.tensor(q, dtype=dt, device="cuda")
        F = torch.empty((N, 3), dtype=dt, device="cuda") if mode == "ik_forces" else None
        phi = torch.empty((N,), dtype=dt, device="cuda") if mode != "energy_only" else None
        Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(10):
            plan.evaluate(xd, qd, F, phi, Ed)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            flush()
            st[i].record()
            plan.evaluate(xd, qd, F, phi, Ed)
            en[i].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / K
        r = {"value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": K,
             "spread_variant": int(plan.params()["spread_variant"])}
        if F is not None:
            r["rel_rms_force_err"] = rel_rms(F.double().cpu().numpy(), Fref)
        out[mode] = r
        plan.close()
    # the ik oracle once on the whole workload (small workloads only)
    if w["M"] <= 64:
        import oracle
        t0 = time.perf_counter()
        oracle.se_kspace_ik(np.asarray(x, np.float64), np.asarray(q, np.float64), w["L"],
                            w["xi"], w["M"], w["P"])
        dt = time.perf_counter() - t0
        out["ik_forces"]["cpu_baseline"] = {"value": 1.0 / dt, "unit": "evals/s",
                                            "cores": oracle.num_threads(), "kind": "oracle",
                                            "sample": "one whole evaluation"}
    return out


def real_space(se, torch, x, q, w, prec, K, flush, plan):
    """The real-space part of the Ewald sum (cell lists, cut-off 1 nm, or L/3
    for boxes under 3 nm) on the same input, alone and after the k-space
    evaluation into the same outputs (the whole Ewald sum)."""
    N = len(q)
    rc = min(1.0, w["L"] / 3.0)
    rprec = "fp64" if prec == "fp64" else "fp32"
    rs = se.RealSpace(N, w["L"], w["xi"], rc, precision=rprec)
    dt = rs.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = {"rc": rc, "cells_per_dim": rs.cells_per_dim(), "precision": rprec}
    # algorithmic work: (2K+1)^3 (rc/K)^3 rho distance tests (8 flops) and
    # (4 pi/3) rc^3 rho pair terms (about 40 flops with the transcendentals)
    nc = rs.cells_per_dim()
    K = max(1, int(round(nc * rc / w["L"])))
    rho = N / w["L"] ** 3
    cand = (2 * K + 1) ** 3 * (w["L"] / nc) ** 3 * rho
    hits = 4.0 / 3.0 * math.pi * rc ** 3 * rho
    flops = N * (8.0 * cand + 40.0 * hits)
    for key, both in (("real_only", False), ("whole_ewald", True)):
        def step():
            if both:
                plan.evaluate(xd, qd, F, phi, Ed)
            rs.evaluate(xd, qd, F, phi, Ed, accumulate=both)
        for _ in range(10):
            step()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            flush()
            st[i].record()
            step()
            en[i].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / K
        out[key] = {"value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": K}
    from paper_1712_04718_gb300 import se as _se
    pk = _se.probe_peak("fp64_fma" if rprec == "fp64" else "fp32_fma") / 1e12
    t = out["real_only"]["ms_per_step"] * 1e-3
    out["roofline"] = {"kernel": "k_rs_pairs (+ count, scan, scatter)", "bound": "alu",
                       "unit": "TFLOP/s", "achieved": flops / t / 1e12, "peak": pk,
                       "frac": flops / t / 1e12 / pk,
                       "work": "N (8 flops x %.0f candidates + 40 flops x %.0f pairs within rc)" % (cand, hits),
                       "peak_source": "measured: se_probe_peak FMA rate (this run)"}
    rs.close()
    # the oracle's real-space image sum at a sample of target atoms, scaled to the box
    import oracle
    ns = min(N, 64)
    idx = np.random.default_rng(0).choice(N, ns, replace=False)
    x64, q64 = np.asarray(x, np.float64), np.asarray(q, np.float64)
    t0 = time.perf_counter()
    oracle.ewald_real_at(x64, q64, w["L"], w["xi"], rc, idx)
    dt = (time.perf_counter() - t0) * N / ns
    out["cpu_baseline"] = {"value": 1.0 / dt, "unit": "evals/s", "cores": oracle.num_threads(),
                           "kind": "oracle", "sample": "%d target atoms of the box (all images "
                           "within rc), scaled to all %d" % (ns, N)}
    return out


def xi_balance(se, torch, x, q, w, prec):
    """The splitting-parameter balance of the paper's Sec. 6.2 on this machine:
    the whole Ewald evaluation (k-space plan, then the real-space sum) timed
    against the real-space cut-off, hence xi, at a fixed rms force tolerance
    of 1e-3 of the box's rms total force, each cut-off with the parameters
    se_select_params gives (tuning.tune_ewald).  The fastest is the balance."""
    from paper_1712_04718_gb300 import tuning
    N = len(q)
    rprec = "fp64" if prec == "fp64" else "fp32"
    dt = torch.float64 if rprec == "fp64" else torch.float32
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
    rs = se.RealSpace(N, w["L"], w["xi"], min(1.0, w["L"] / 3.0), precision=rprec)
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.evaluate(xd, qd, F, phi, Ed)
    rs.evaluate(xd, qd, F, phi, Ed, accumulate=True)
    f_rms = float(torch.sqrt((F.double() ** 2).sum(1).mean()))
    plan.close()
    rs.close()
    tol = 1e-3 * f_rms
    best, table = tuning.tune_ewald(xd, qd, w["L"], tol, precision=rprec)
    return {"tol_rel_to_rms_force": 1e-3, "tol_abs": tol, "best": best, "table": table,
            "note": "se_select_params sizes each error source to tol (the paper's estimates)"}


def no_graph(se, torch, plan, xd, qd, F, phi, Ed, flush, K):
    """The headline loop with every kernel launched directly (no CUDA graph)."""
    plan.set_graph(False)
    for _ in range(5):
        plan.evaluate(xd, qd, F, phi, Ed)
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for i in range(K):
        flush()
        st[i].record()
        plan.evaluate(xd, qd, F, phi, Ed)
        en[i].record()
    torch.cuda.synchronize()
    plan.set_graph(True)
    ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / K
    return {"value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": K}


def e2e(se, torch, x, q, w, prec, K, cfg):
    """Host buffers through se_energy_force_host: H2D of xyz and q, the
    evaluation, D2H of F, phi and E, every step."""
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
    if prec != "fp64":
        plan.set_tuning(*cfg)
    dt = plan.dtype
    hx = torch.tensor(x, dtype=dt).pin_memory()
    hq = torch.tensor(q, dtype=dt).pin_memory()
    hF = torch.empty((N, 3), dtype=dt).pin_memory()
    hphi = torch.empty((N,), dtype=dt).pin_memory()
    args = (hx.data_ptr(), hq.data_ptr(), hF.data_ptr(), hphi.data_ptr())
    for _ in range(5):
        plan.energy_force_host_ptrs(*args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        plan.energy_force_host_ptrs(*args)
    t1 = time.perf_counter()
    plan.close()
    es = hx.element_size()
    return {"value": K / (t1 - t0), "unit": "evals/s", "steps": K,
            "h2d_bytes_per_step": N * 4 * es, "d2h_bytes_per_step": N * 4 * es + 8 + 32,
            "timing": "host wall clock around each synchronous call"}


def cpu_baseline(x, q, w, seconds):
    """The FP64 CPU oracle (plain SE, O2) on the host cores: whole evaluations of
    the same workload, repeated for about `seconds`."""
    import oracle
    xd, qd = np.asarray(x, np.float64), np.asarray(q, np.float64)
    cm = 64 if w["prec"] == "fp64" else 32
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.se_kspace(xd, qd, w["L"], w["xi"], w["M"], w["P"], cell_mode=cm)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (n >= 3 and el * (n + 1) / n > 3 * seconds):
            break
    return {"value": n / el, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d whole evaluations of %s by the FP64 CPU SE oracle (direct exp, direct "
                      "DFT), %.1f s" % (n, "the workload", el)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle (plain SE) on the host cores."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    x, q, w, prec = workload(args.workload)
    xd, qd = np.asarray(x, np.float64), np.asarray(q, np.float64)
    cm = 64 if w["prec"] == "fp64" else 32
    t0 = time.perf_counter()
    oracle.se_kspace(xd, qd, w["L"], w["xi"], w["M"], w["P"], cell_mode=cm)
    t1 = time.perf_counter()
    one = t1 - t0
    budget = 150.0
    W = args.warmup if one * (args.warmup + args.steps) <= budget else min(args.warmup, 1)
    for _ in range(max(0, W - 1)):
        oracle.se_kspace(xd, qd, w["L"], w["xi"], w["M"], w["P"], cell_mode=cm)
    K = args.steps
    run = K if one * K <= budget else max(1, int(budget / one))
    t0 = time.perf_counter()
    for _ in range(run):
        oracle.se_kspace(xd, qd, w["L"], w["xi"], w["M"], w["P"], cell_mode=cm)
    el = time.perf_counter() - t0
    value = run / el
    N = len(q)
    sample = ("%d whole evaluations of the workload (of %d requested steps) by the FP64 CPU SE "
              "oracle" % (run, K))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": ws, "steps": K, "warmup": args.warmup, "ms_per_step": el / run * 1e3,
        "ns_per_atom": el / run * 1e9 / N, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "L": w["L"], "xi": w["xi"], "M": w["M"],
                   "P": w["P"], "precision": w["prec"]},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
