#!/usr/bin/env python3
"""Benchmark of the SE k-space path: energy+force evaluations per second at
each workload's stated relative rms force error.

One step = one whole k-space evaluation (bin, spread, FFT, scale, inverse
FFT, gather; energy, forces and potentials) of the named workload, with the
inputs resident on the GPU.  Between timed steps L2 is flushed by writing a
256 MiB buffer (outside the timed events).  `e2e` times the same evaluation
through the host-buffer entry point (se_energy_force_host: copies in,
compute, copies out).

The headline is the 21 642-atom water box at P = 8, the smallest even
support at which that box meets its stated error of 1e-3 (P = 6, the stated
support, gives 3e-3; it is measured as a leg).  After the headline, one
compact leg per other workload (`legs`, last key of the line): its rate,
error against the direct Ewald sum, target, roofline fraction and clocks;
the single-precision legs also time the plain FP64 GPU pipeline at the
smallest even P that is at least as accurate (`fp64_eq`).

Every stated error is the relative rms force error against O1, the FP64
CPU direct Ewald k-space sum, at 256 sampled atoms (for the ensembles, at
sampled atoms of 8 sampled systems).  O1 runs inside the cpu_baseline leg,
which times it beside O2 (the plain FP64 CPU SE) with all cores and with one
thread: the oracle's outputs of that leg are the reference of the error
statement.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--legs all|none|NAME,...] [--extras FILE]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

With torchrun (N > 1) every rank evaluates its own replica of the workload
(the path does not shard a single system; legs are skipped); value = all
ranks' evaluations per second of the slowest rank.  An ensemble workload is
sharded over the ranks by system (paper_1712_04718_gb300.sharding).
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

DEFAULT_WORKLOAD = "water-L6-M52-P8-fp32comp"
LEG_WORKLOADS = ("uniform-1000-L3-M32-P16-fp64", "water-L6-M52-P6-fp32comp",
                 "water-L6-M96-P24-fp64", "water-L10-M84-P8-fp32comp",
                 "ensemble-64-water-L3to7-P8-fp32comp", "ensemble-64-water-L3to7-P10-fp32comp")
METRIC = "SE k-space energy+force evals/s and ns/atom at stated rms force error vs FP64"
O1_SAMPLE = 256          # sampled atoms of the error statement
ENS_SAMPLE_SYSTEMS = 8   # sampled systems of an ensemble's error statement


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--legs", default="all",
                    help="workloads measured after the headline: all, none, or a comma list")
    ap.add_argument("--cpu-seconds", type=float, default=4.0,
                    help="bounded CPU work of each timing of the cpu_baseline leg")
    ap.add_argument("--extras", default="",
                    help="also run the legs beyond the metric (evaluation modes, real space, "
                         "xi balance, no-graph, unsorted spread, per-stage events, cost model) "
                         "and write them to this JSON file")
    ap.add_argument("--bare", action="store_true",
                    help="time the headline steps only (no stage times, legs, oracle or e2e): "
                         "the command of the ncu launch lists")
    ap.add_argument("--tile", type=int, default=0,
                    help="spreading tile edge (0 = autotune, JSON-cached)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="spread variant (-1 = autotune with the tile; 3 sorted, 4 unsorted)")
    return ap.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def r4(v):
    """v rounded to 4 significant digits (floats only), for a compact line."""
    if isinstance(v, float) and math.isfinite(v) and v != 0.0:
        return float("%.4g" % v)
    return v


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
        return self

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


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def unit_peaks(se, peaks):
    """Peaks of the units the kernels are bound by.  The FP32 FMA rate and
    the shared-memory atomic rate are derived from unit counts and the
    maximum SM clock: 152 SMs x 128 FP32 lanes x 2 flops, and 152 SMs x 32
    banks (one 32-bit atomic per bank and clock); FP64 is GB300's nominal
    1.25 TFLOP/s; HBM is the measured copy bandwidth.  The rates the
    library's own probe kernels reach on this GPU (se_probe_peak) are given
    beside them."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return {
        "fp32_fma_tflops": 152 * 128 * 2 * mhz * 1e6 / 1e12,
        "fp64_fma_tflops": 1.25,
        "smem_atomic_gops": 152 * 32 * mhz * 1e6 / 1e9,
        "hbm_gbs": peaks.get("hbm_gbs", 6800.0),
        "hbm_source": "measured (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "fallback",
        "probe": {"fp32_fma_tflops": se.probe_peak("fp32_fma") / 1e12,
                  "fp64_fma_tflops": se.probe_peak("fp64_fma") / 1e12,
                  "smem_atomic_u32_gops": se.probe_peak("smem_atomic_u32") / 1e9},
    }


def make_flush(torch):
    flush_w = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def flush():
        # write 256 MiB (evicts everything), then read another 256 MiB so that
        # the dirty lines are written back before the timed step starts
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_out)
    return flush


def time_steps(torch, step, K, W, flush, min_seconds=0.0, ws=1):
    """W untimed warm-up steps, then K (at least enough for min_seconds)
    timed steps with L2 flushed before each, CUDA events around each step on
    the launching stream, nvidia-smi clocks sampled meanwhile.  Returns
    (total ms of the timed steps, K, clocks)."""
    for _ in range(max(3, W)):
        flush()
        step()
    torch.cuda.synchronize()
    if min_seconds > 0:
        t0 = time.perf_counter()
        for _ in range(5):
            flush()
            step()
        torch.cuda.synchronize()
        per = (time.perf_counter() - t0) / 5
        K = max(K, int(math.ceil(min_seconds / max(per, 1e-6))))
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device()).start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(K):
        flush()
        st[i].record()
        step()
        en[i].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    return sum(a.elapsed_time(b) for a, b in zip(st, en)), K, clk


def graph_time_us(torch, fn, reps=20, iters=10):
    """Average device time (us) of one call of fn: fn launched `reps` times
    back to back into one CUDA graph, the graph replayed `iters` times
    between two CUDA events on the launching stream (no launch gaps)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(iters):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    del g
    return ms * 1e3 / (iters * reps)


def stage_times_us(torch, plan, xd, qd, F, phi, Ed):
    """Device time of the three stages of one evaluation from CUDA-graph
    replays: transform = se_scale (forward transform, scaling, inverse
    transform), spread = (se_spread + se_scale) - transform (the spread's
    grid is consumed by the transform, so it is not replayed alone), gather =
    se_gather.  The gather is one kernel launch."""
    t_tr = graph_time_us(torch, lambda: plan.scale(None))

    def sp_tr():
        plan.spread(xd, qd)
        plan.scale(None)
    t_sptr = graph_time_us(torch, sp_tr)
    t_ga = graph_time_us(torch, lambda: plan.gather(xd, qd, phi, F, Ed))
    # leave the plan with a complete evaluation
    plan.evaluate(xd, qd, F, phi, Ed)
    torch.cuda.synchronize()
    return {"spread": max(0.0, t_sptr - t_tr), "transform": t_tr, "gather": t_ga}


def dft_split(M):
    """M1 of the factored transforms: the largest divisor of M not above sqrt(M)."""
    best, a = 1, 2
    while a * a <= M:
        if M % a == 0:
            best = a
        a += 1
    return best


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


def kernel_sources_sha():
    """Digest of the kernel sources (a profile's DRAM figures apply only to
    the sources they were taken on)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("se_fast.cuh", "se_fast_launch.cuh", "se_kernels.cuh", "se_dft.cuh",
              "se_internal.h"):
        with open(os.path.join(ROOT, "paper_1712_04718_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload_name):
    """DRAM bytes per launch (read + write) of `kernel` on `workload_name`
    from the data file profiles/traffic.json, written from one ncu capture:
    {workload: {"kernel_sources_sha256": ..., "dram_bytes_per_launch":
    {kernel: bytes}, "source": ...}}.  None when the file holds no figure
    for the kernel or the figure was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None, None
    rec = data.get(workload_name)
    if not rec or rec.get("kernel_sources_sha256") != kernel_sources_sha():
        return None, None
    v = rec.get("dram_bytes_per_launch", {}).get(kernel)
    if v is None:
        return None, None
    return float(v), rec.get("source")


def roofline(kind, amount, kernel, us, prec, up, workload_name):
    """Roofline object of one kernel: algorithmic work per launch over its
    average launch duration (us), against the peak of its bounding unit."""
    secs = us * 1e-6
    if kind == "smem_atomic":
        r = {"bound": "alu", "unit": "Gop/s", "achieved": amount / secs / 1e9,
             "peak": up["smem_atomic_gops"],
             "peak_source": "152 SMs x 32 shared-memory atomics/clock x max SM clock",
             "probe_peak": up["probe"]["smem_atomic_u32_gops"]}
    elif kind == "flop":
        fp64 = prec == "fp64"
        r = {"bound": "alu", "unit": "TFLOP/s", "achieved": amount / secs / 1e12,
             "peak": up["fp64_fma_tflops"] if fp64 else up["fp32_fma_tflops"],
             "peak_source": ("GB300 nominal FP64 rate" if fp64 else
                             "152 SMs x 128 FP32 lanes x 2 flops x max SM clock"),
             "probe_peak": up["probe"]["fp64_fma_tflops" if fp64 else "fp32_fma_tflops"]}
    else:
        r = {"bound": "hbm", "unit": "GB/s", "achieved": amount / secs / 1e9,
             "peak": up["hbm_gbs"], "peak_source": up["hbm_source"]}
    traffic, tsrc = profiled_traffic(kernel, workload_name)
    r.update({"kernel": kernel, "frac": r["achieved"] / r["peak"], "traffic": traffic,
              "traffic_source": tsrc, "work_per_launch": amount, "launch_us": us,
              "launch_us_source": "CUDA-graph replay of back-to-back launches, CUDA events"})
    return {k: r4(v) for k, v in r.items()}


def rel_rms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


# ---------------------------------------------------------------------------
# cpu_baseline leg: the FP64 CPU oracle on the host cores (bounded samples).
# O2 (plain SE) with all cores and with one thread, and O1 (the direct Ewald
# k-space sum) at sampled atoms; O1's forces there are also the reference of
# the error statements (nothing else in this file runs the oracle).

def o1_tolerance(target):
    """k-vector cut-off of O1 for a workload held to `target`: modes with
    e^{-k^2/(4 xi^2)} < tol are left out, tol = target^2 (at most 1e-6, at
    least 1e-16), far below the error being measured."""
    return max(1e-16, min(1e-6, target * target))


def o1_sample(x, q, L, xi, target, nsample=O1_SAMPLE, seed=0):
    """O1 at nsample seeded atoms: the structure factor over all atoms, then
    phi and F at the sample.  Returns (idx, F [n, 3], seconds)."""
    import oracle
    x64, q64 = np.asarray(x, np.float64), np.asarray(q, np.float64)
    N = len(q64)
    idx = np.sort(np.random.default_rng(seed).choice(N, min(N, nsample), replace=False))
    nmax = oracle.nmax_for(xi, L, o1_tolerance(target))
    t0 = time.perf_counter()
    S = oracle.ewald_structure(x64, q64, L, nmax)
    _, F = oracle.ewald_eval(x64[idx], q64[idx], S, L, xi, nmax)
    return idx, F, time.perf_counter() - t0, nmax


def o2_rate(x, q, L, xi, M, P, cm, seconds, threads=0):
    """O2 whole evaluations per second for about `seconds` (at least one),
    with `threads` OpenMP threads (0 = all)."""
    import oracle
    xd, qd = np.asarray(x, np.float64), np.asarray(q, np.float64)
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        n, t0 = 0, time.perf_counter()
        while True:
            oracle.se_kspace(xd, qd, L, xi, M, P, cell_mode=cm)
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds or (n >= 2 and el * (n + 1) / n > 3 * seconds):
                break
        used = oracle.num_threads()
    finally:
        oracle.set_num_threads(all_threads)
    return n / el, n, el, used


def cpu_baseline_leg(x, q, w, seconds, one_thread=True):
    """The cpu_baseline object of a single-system workload, and O1's sample
    (idx, F) for the error statement."""
    import oracle
    oracle.build()
    cm = 64 if w["prec"] == "fp64" else 32
    v, n, el, cores = o2_rate(x, q, w["L"], w["xi"], w["M"], w["P"], cm, seconds)
    out = {"value": r4(v), "unit": "evals/s", "cores": cores, "kind": "oracle",
           "sample": "%d whole evaluations by the FP64 CPU SE oracle (O2: direct exp, direct "
                     "DFT), %.1f s" % (n, el)}
    if one_thread:
        v1, n1, el1, _ = o2_rate(x, q, w["L"], w["xi"], w["M"], w["P"], cm, seconds, threads=1)
        out["one_thread"] = {"value": r4(v1), "cores": 1,
                             "sample": "%d whole evaluations, %.1f s" % (n1, el1)}
    idx, F1, t1, nmax = o1_sample(x, q, w["L"], w["xi"], w["target_rel_force_err"])
    N = len(q)
    out["o1"] = {"seconds": r4(t1), "cores": cores, "targets": len(idx), "nmax": nmax,
                 "kind": "direct Ewald k-space sum (structure factor over all atoms, "
                         "then the sampled atoms)"}
    return out, (idx, F1)


# ---------------------------------------------------------------------------
# Single-system workloads

def setup_plan(se, torch, tuning, x, q, w, prec, P=None, tile=0, variant=-1):
    N = len(q)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], P or w["P"], precision=prec)
    dt = plan.dtype
    xd = torch.tensor(np.asarray(x), dtype=dt, device="cuda")
    qd = torch.tensor(np.asarray(q), dtype=dt, device="cuda")
    if tile or variant >= 0:
        plan.set_tuning(max(0, variant), tile)
    elif prec != "fp64":
        tuning.tune_plan(plan, xd, qd)
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    return plan, xd, qd, F, phi, Ed


# "Equal accuracy": an error within 1 % of the single-precision run's.  The
# two differ by rounding only when the approximation error dominates (the
# same P), and the 256-atom estimate of an rms error is itself good to a
# few per cent, so a finer split would pick P by noise.
EQUAL_ACCURACY_BAND = 1.01


def fp64_equal_accuracy(se, torch, tuning, x, q, w, err32, ref, K, W, flush):
    """The plain FP64 GPU pipeline on the same positions at the smallest even
    P (from the workload's own) whose error against O1 is at most the
    single-precision run's (within EQUAL_ACCURACY_BAND); timed like the
    headline."""
    idx, F1 = ref
    for P in range(w["P"], w["P"] + 10, 2):
        if P > w["M"]:
            break
        plan, xd, qd, F, phi, Ed = setup_plan(se, torch, tuning, np.asarray(x, np.float64),
                                              np.asarray(q, np.float64), w, "fp64", P=P)
        plan.evaluate(xd, qd, F, phi, Ed)
        torch.cuda.synchronize()
        err = rel_rms(F.cpu().numpy()[idx], F1)
        if err > EQUAL_ACCURACY_BAND * err32 and P + 2 < w["P"] + 10:
            plan.close()
            continue
        ms, k, _ = time_steps(torch, lambda: plan.evaluate(xd, qd, F, phi, Ed), K, W, flush)
        plan.close()
        return {"P": P, "value": r4(k / (ms / 1e3)), "ms": r4(ms / k),
                "err": r4(err), "equal": err <= EQUAL_ACCURACY_BAND * err32}
    return None


def run_single(args, se, torch, name, K, W, flush, up, headline=False, ws=1):
    """One single-system workload: rate, error against O1, roofline,
    clocks; the FP64 equal-accuracy run for single-precision workloads."""
    from paper_1712_04718_gb300 import systems, tuning
    x, q, w = systems.make(name)
    prec = "fp64" if w["prec"] == "fp64" else "fp32"
    N = len(q)
    plan, xd, qd, F, phi, Ed = setup_plan(se, torch, tuning, x, q, w, prec,
                                          tile=args.tile if headline else 0,
                                          variant=args.variant if headline else -1)
    variant = int(plan.params()["spread_variant"])
    tile = int(plan.params()["tile"])
    step = lambda: plan.evaluate(xd, qd, F, phi, Ed)   # noqa: E731
    total_ms, K, clk = time_steps(torch, step, K, W, flush,
                                  min_seconds=0.0 if headline else 0.3, ws=ws)
    total_ms_max = total_ms
    if ws > 1:
        from paper_1712_04718_gb300.sharding import max_over_ranks
        total_ms_max = max_over_ranks(total_ms, ws, "cuda")
    ms_step = total_ms_max / K
    res = {"workload": name, "N": N, "w": w, "prec": prec, "variant": variant, "tile": tile,
           "K": K, "ms_step": ms_step, "value": ws * K / (total_ms_max / 1e3), "clocks": clk,
           "x": x, "q": q}
    # per-stage device times (graph replays) and the roofline of the gather
    st = stage_times_us(torch, plan, xd, qd, F, phi, Ed)
    work = stage_work(w, prec, N, variant, tile)
    kind, amount, kname = work["gather"]
    res["stages_us"] = st
    res["roofline"] = roofline(kind, amount, kname, st["gather"], prec, up, name)
    res["dominant"] = max(st, key=st.get)
    res["F"] = F.double().cpu().numpy()
    res["plan_cfg"] = (variant, tile)
    if headline and ws == 1:
        res["e2e"] = e2e(se, torch, x, q, w, prec, max(20, min(K, 500)), (variant, tile))
    if name == "water-L10-M84-P8-fp32comp" and ws == 1:
        res["autograd"] = autograd_timing(se, torch, x, q, w, prec, plan, xd, qd,
                                          max(20, min(K, 200)), flush)
    plan.close()
    return res


def finish_single(args, se, torch, res, K, W, flush, headline):
    """cpu_baseline leg (with the O1 sample), the error statement and the
    FP64 equal-accuracy run of a measured single-system workload."""
    from paper_1712_04718_gb300 import tuning
    w = res["w"]
    cb, ref = cpu_baseline_leg(res["x"], res["q"], w, args.cpu_seconds if headline else 2.0,
                               one_thread=True)
    idx, F1 = ref
    err = rel_rms(res["F"][idx], F1)
    acc = {"rel_rms_force_err": r4(err), "target": w["target_rel_force_err"],
           "target_source": w["target_source"], "target_met": err <= w["target_rel_force_err"],
           "reference": "O1 (FP64 CPU direct Ewald k-space sum) at %d sampled atoms" % len(idx)}
    eq = None
    if res["prec"] != "fp64":
        eq = fp64_equal_accuracy(se, torch, tuning, res["x"], res["q"], w, err, ref,
                                 max(50, min(K, 500)), W, flush)
    return cb, acc, eq


def e2e(se, torch, x, q, w, prec, K, cfg):
    """Host buffers through se_energy_force_host, every step: xyz and q from
    page-locked host memory to the GPU, the evaluation, F, phi and E back to
    host memory.  With these (mapped) buffers the library's kernels read the
    inputs and write the outputs in host memory directly over the host link,
    as one CUDA graph; the bytes counted are those that cross the link."""
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
    return {"value": r4(K / (t1 - t0)), "unit": "evals/s", "steps": K,
            "h2d_bytes_per_step": N * 4 * es, "d2h_bytes_per_step": N * 4 * es + 8 + 32,
            "timing": "host wall clock around each synchronous call",
            "transfer": "kernels read and write the pinned, mapped host buffers directly"}


def autograd_timing(se, torch, x, q, w, prec, plan, xd, qd, K, flush):
    """The differentiable energy (autograd.se_energy): forward alone (spread
    and scaling, energy from the grid) and forward + backward (the adjoint
    gather: dE/dx, dE/dq), each step launched from Python through
    torch.autograd (eager: the autograd engine's host time is part of it),
    and the forward + backward replayed as one captured CUDA graph; timed
    with CUDA events around the step."""
    from paper_1712_04718_gb300.autograd import se_energy
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
        ms, k, _ = time_steps(torch, fn, K, 5, flush)
        res[name] = r4(k / (ms / 1e3))
    # the same forward + backward captured in one CUDA graph (static inputs),
    # the way a training step hides the autograd engine's host time
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            fwd_bwd()
    torch.cuda.current_stream().wait_stream(s)
    xg.grad = None
    qg.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        se_energy(xg, qg, plan).backward()
    ms, k, _ = time_steps(torch, g.replay, K, 5, flush)
    res["forward_backward_graph"] = r4(k / (ms / 1e3))
    del g
    res["unit"] = "evals/s"
    return res


# ---------------------------------------------------------------------------
# Ensembles

def ensemble_sample(ens):
    """ENS_SAMPLE_SYSTEMS systems spread over the box sizes (the smallest and
    the largest included)."""
    order = sorted(range(len(ens)), key=lambda i: ens[i]["L"])
    k = min(len(ens), ENS_SAMPLE_SYSTEMS)
    return sorted({order[round(j * (len(order) - 1) / max(1, k - 1))] for j in range(k)})


def run_ensemble_workload(args, se, torch, name, K, W, flush, up, headline=False, ws=1, rank=0):
    from paper_1712_04718_gb300 import sharding, systems, tuning
    w = systems.WORKLOADS[name]
    ens = systems.ensemble(S=w["S"], spacing=w["spacing"])
    mine_idx = sharding.shard([len(d["q"]) for d in ens], [d["M"] for d in ens], w["P"], ws, rank)
    mine = [ens[i] for i in mine_idx]
    Ns = [len(d["q"]) for d in mine]
    b = se.Batch(Ns, [d["L"] for d in mine], [d["M"] for d in mine], w["xi"], w["P"])
    xd = torch.tensor(np.concatenate([d["x"] for d in mine]), device="cuda")
    qd = torch.tensor(np.concatenate([d["q"] for d in mine]), device="cuda")
    if headline and args.tile:
        b.set_tile(args.tile)
        tile = args.tile
    else:
        tile, _, _ = tuning.tune_batch(b, xd, qd)
    Ntot = int(sum(Ns))
    F = torch.empty((Ntot, 3), dtype=torch.float32, device="cuda")
    phi = torch.empty((Ntot,), dtype=torch.float32, device="cuda")
    E = torch.empty((len(mine),), dtype=torch.float64, device="cuda")
    step = lambda: b.evaluate(xd, qd, F, phi, E)   # noqa: E731
    total_ms, K, clk = time_steps(torch, step, K, W, flush,
                                  min_seconds=0.0 if headline else 0.3, ws=ws)
    if ws > 1:
        total_ms = sharding.max_over_ranks(total_ms, ws, "cuda")
    ms_step = total_ms / K
    Nall = sum(len(d["q"]) for d in ens)
    res = {"workload": name, "w": w, "K": K, "ms_step": ms_step, "value": K / (total_ms / 1e3),
           "clocks": clk, "Nall": Nall, "tile": tile, "systems": len(ens),
           "M_range": [min(d["M"] for d in ens), max(d["M"] for d in ens)]}
    # per-stage times: CUDA events between the stages of direct launches
    # (each stage runs for hundreds of microseconds here, far above the
    # launch rate), and the roofline of the larger of spread and gather
    b.set_timing(True)
    for _ in range(20):
        b.evaluate(xd, qd, F, phi, E)
    torch.cuda.synchronize()
    stages, nst = b.get_timing()
    b.set_timing(False)
    us = {k: v / max(1, nst) * 1e3 for k, v in stages.items()}
    res["stages_us"] = us
    P3 = float(w["P"]) ** 3
    if us["spread"] >= us["gather"]:
        roof = {"kernel": "k_bspread", "bound": "alu", "unit": "Gop/s",
                "achieved": Ntot * P3 / (us["spread"] * 1e-6) / 1e9, "peak": up["smem_atomic_gops"],
                "work_per_launch": Ntot * P3, "launch_us": us["spread"]}
    else:
        roof = {"kernel": "k_bgather_tile / k_bgather", "bound": "alu", "unit": "TFLOP/s",
                "achieved": 4.0 * Ntot * P3 / (us["gather"] * 1e-6) / 1e12,
                "peak": up["fp32_fma_tflops"], "work_per_launch": 4.0 * Ntot * P3,
                "launch_us": us["gather"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["launch_us_source"] = "CUDA events between the stages of direct launches"
    res["roofline"] = {k: r4(v) for k, v in roof.items()}
    res["F"] = F.double().cpu().numpy()
    res["offsets"] = np.concatenate([[0], np.cumsum(Ns)])
    res["ens"], res["mine_idx"] = ens, mine_idx
    if headline and ws == 1:
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
        res["e2e"] = {"value": r4(k2 / (t1 - t0)), "unit": "ensemble evals/s", "steps": k2,
                      "h2d_bytes_per_step": hx.numel() * 4 + hq.numel() * 4,
                      "d2h_bytes_per_step": hF.numel() * 4 + hE.numel() * 8}
    b.close()
    return res


_ENS_O1 = {}


def ensemble_cpu_baseline(res, seconds):
    """cpu_baseline leg of an ensemble: O2 over whole systems in order until
    `seconds` (scaled by atoms to the ensemble), and O1 at sampled atoms of
    the sampled systems (kept for the error statement; shared between the
    ensembles of one box set, whose positions are the same)."""
    import oracle
    oracle.build()
    w, ens = res["w"], res["ens"]
    t0 = time.perf_counter()
    n_done, k_sys = 0, 0
    for d in ens:
        oracle.se_kspace(np.asarray(d["x"], np.float64), np.asarray(d["q"], np.float64),
                         d["L"], w["xi"], d["M"], w["P"], cell_mode=32)
        n_done += len(d["q"])
        k_sys += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = (time.perf_counter() - t0) * res["Nall"] / n_done
    cb = {"value": r4(1.0 / dt), "unit": "ensemble evals/s", "cores": oracle.num_threads(),
          "kind": "oracle", "sample": "O2 on the first %d of %d systems (%d atoms), scaled by "
                                      "atoms" % (k_sys, len(ens), n_done)}
    sample = ensemble_sample(ens)
    refs, t_o1 = {}, 0.0
    for s in sample:
        key = (len(ens), s, w["target_rel_force_err"])
        if key not in _ENS_O1:
            d = ens[s]
            idx, F1, t1, _ = o1_sample(d["x"], d["q"], d["L"], w["xi"], w["target_rel_force_err"],
                                       nsample=O1_SAMPLE, seed=s)
            _ENS_O1[key] = (idx, F1, t1)
        refs[s] = _ENS_O1[key][:2]
        t_o1 += _ENS_O1[key][2]
    cb["o1"] = {"seconds": r4(t_o1), "systems": len(sample), "targets_per_system": O1_SAMPLE,
                "kind": "direct Ewald k-space sum"}
    return cb, refs


def ensemble_errors(res, refs):
    """Relative rms force error against O1 of each sampled system."""
    errs = {}
    pos = {s: j for j, s in enumerate(res["mine_idx"])}
    off = res["offsets"]
    for s, (idx, F1) in refs.items():
        if s not in pos:
            continue
        j = pos[s]
        errs[s] = rel_rms(res["F"][off[j]:off[j + 1]][idx], F1)
    return errs


def ensemble_fp64_equal(se, torch, res, refs, err32, K, W, flush):
    """The plain FP64 GPU pipeline on every system of the ensemble (one FP64
    plan per system, each evaluation replayed as its plan's CUDA graph) at
    the smallest even P (from the ensemble's own) whose largest error over
    the sampled systems is at or below the single-precision batch's."""
    w, ens = res["w"], res["ens"]
    for P in range(w["P"], w["P"] + 10, 2):
        plans = []
        for d in ens:
            N = len(d["q"])
            p = se.Plan(N, d["L"], w["xi"], d["M"], P, precision="fp64")
            xd = torch.tensor(np.asarray(d["x"], np.float64), device="cuda")
            qd = torch.tensor(np.asarray(d["q"], np.float64), device="cuda")
            F = torch.empty((N, 3), dtype=torch.float64, device="cuda")
            phi = torch.empty((N,), dtype=torch.float64, device="cuda")
            Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
            plans.append((p, xd, qd, F, phi, Ed))

        def step():
            for p, xd, qd, F, phi, Ed in plans:
                p.evaluate(xd, qd, F, phi, Ed)
        step()
        torch.cuda.synchronize()
        err = max(rel_rms(plans[s][3].cpu().numpy()[idx], F1) for s, (idx, F1) in refs.items())
        if err > EQUAL_ACCURACY_BAND * err32 and P + 2 < w["P"] + 10:
            for t in plans:
                t[0].close()
            continue
        ms, k, _ = time_steps(torch, step, K, W, flush)
        for t in plans:
            t[0].close()
        return {"P": P, "value": r4(k / (ms / 1e3)), "ms": r4(ms / k), "err": r4(err),
                "equal": err <= EQUAL_ACCURACY_BAND * err32,
                "form": "one FP64 plan per system, each replayed as its CUDA graph"}
    return None


# ---------------------------------------------------------------------------
# Output

def compact_leg(res, acc, eq):
    """One leg of the line: rate, time, error, target, roofline, clocks."""
    leg = {"w": res["workload"], "value": r4(res["value"]),
           "unit": "ensemble evals/s" if "Nall" in res else "evals/s",
           "ms": r4(res["ms_step"]),
           "ns_atom": r4(res["ms_step"] * 1e6 / res.get("Nall", res.get("N", 1))),
           "err": acc["rel_rms_force_err"], "target": acc["target"], "met": acc["target_met"],
           "frac": res["roofline"]["frac"], "kernel": res["roofline"]["kernel"],
           "sm_mhz": res["clocks"].get("sm_mhz"), "thr": res["clocks"].get("reasons")}
    if eq:
        leg["fp64_eq"] = eq
    if "autograd" in res:
        leg["autograd"] = res["autograd"]
    return leg


def run_leg(args, se, torch, name, K, W, flush, up):
    if name.startswith("ensemble"):
        res = run_ensemble_workload(args, se, torch, name, K, W, flush, up)
        cb, refs = ensemble_cpu_baseline(res, 2.0)
        errs = ensemble_errors(res, refs)
        e32 = max(errs.values())
        w = res["w"]
        acc = {"rel_rms_force_err": r4(e32), "target": w["target_rel_force_err"],
               "target_met": e32 <= w["target_rel_force_err"]}
        eq = ensemble_fp64_equal(se, torch, res, refs, e32, max(10, min(K, 50)), 3, flush)
        return compact_leg(res, acc, eq)
    res = run_single(args, se, torch, name, K, W, flush, up)
    res["N"] = len(res["q"])
    cb, acc, eq = finish_single(args, se, torch, res, K, W, flush, headline=False)
    return compact_leg(res, acc, eq)


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
    flush = make_flush(torch)
    K, W = args.steps, args.warmup
    name = args.workload
    if args.bare:
        return run_bare(args, se, torch, name, K, W, flush, ws, rank)
    peaks = measured_peaks()
    up = unit_peaks(se, peaks)
    ens = name.startswith("ensemble")
    if ens:
        res = run_ensemble_workload(args, se, torch, name, K, W, flush, up, headline=True,
                                    ws=ws, rank=rank)
        N = res["Nall"]
        unit = "ensemble evals/s"
        config = {"workload": name, "systems": res["systems"], "atoms": N,
                  "M_range": res["M_range"], "P": res["w"]["P"], "xi": res["w"]["xi"],
                  "precision": res["w"]["prec"],
                  "parallelism": "systems sharded over ranks" if ws > 1 else "single",
                  "spread_tile": res["tile"], "pipeline": "batched, one CUDA graph",
                  "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)"}
        launches = 8
        dtype = "f32"
    else:
        res = run_single(args, se, torch, name, K, W, flush, up, headline=True, ws=ws)
        w = res["w"]
        N = len(res["q"])
        res["N"] = N
        unit = "evals/s"
        variant, tile = res["variant"], res["tile"]
        config = {"workload": name, "N": N, "L": w["L"], "xi": w["xi"], "M": w["M"], "P": w["P"],
                  "precision": w["prec"], "parallelism": "replicas" if ws > 1 else "single",
                  "spread_variant": variant, "spread_tile": tile if variant != 4 else None,
                  "pipeline": {3: "single-precision, no cuFFT, sorted spread",
                               4: "single-precision, no cuFFT, unsorted spread"}.get(variant, "cuFFT"),
                  "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)"}
        launches = {3: 6, 4: 5}.get(variant, 5)
        dtype = "f64" if res["prec"] == "fp64" else "f32"
    out = {
        "metric": METRIC, "value": res["value"], "unit": unit, "n_gpus": ws, "steps": res["K"],
        "warmup": W, "ms_per_step": res["ms_step"], "ns_per_atom": res["ms_step"] * 1e6 / N,
        "higher_is_better": True, "scaling": "strong" if ens else "weak", "vs_baseline": None,
        "dtype": dtype, "data": "synthetic", "config": config,
        "roofline": res["roofline"], "clocks": res["clocks"],
        "gpu_launches": launches * res["K"],
        "gpu_launches_note": "own kernels per step: %d" % launches,
    }
    if "stages_us" in res:
        out["stages_us"] = {k: r4(v) for k, v in res["stages_us"].items()}
    if rank == 0 and ws == 1:
        if "e2e" in res:
            out["e2e"] = res["e2e"]
        if ens:
            cb, refs = ensemble_cpu_baseline(res, args.cpu_seconds)
            errs = ensemble_errors(res, refs)
            e32 = max(errs.values())
            acc = {"rel_rms_force_err": r4(e32), "target": res["w"]["target_rel_force_err"],
                   "target_met": e32 <= res["w"]["target_rel_force_err"],
                   "reference": "O1 at %d sampled atoms of %d sampled systems (max over systems)"
                                % (O1_SAMPLE, len(refs))}
            eq = ensemble_fp64_equal(se, torch, res, refs, e32, max(10, min(K, 50)), 3, flush)
        else:
            cb, acc, eq = finish_single(args, se, torch, res, K, W, flush, headline=True)
        out["cpu_baseline"] = cb
        out["accuracy"] = acc
        if eq:
            out["fp64_equal_accuracy"] = eq
        if args.extras:
            extras = run_extras(args, se, torch, res, flush)
            with open(args.extras, "w") as f:
                json.dump(extras, f, indent=1)
        legs = []
        names = (LEG_WORKLOADS if args.legs == "all" else
                 () if args.legs == "none" else tuple(args.legs.split(",")))
        for leg in names:
            if leg == name:
                continue
            try:
                legs.append(run_leg(args, se, torch, leg, max(50, min(K, 500)), W, flush, up))
            except Exception as e:   # a leg that fails is reported, the line still prints
                legs.append({"w": leg, "error": "%s: %s" % (type(e).__name__, str(e)[:120])})
        out["legs"] = legs
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_bare(args, se, torch, name, K, W, flush, ws, rank):
    """The headline's warm-up and timed steps alone (single-system
    workloads), with no other launches: what a launch list under ncu sees."""
    from paper_1712_04718_gb300 import systems, tuning
    x, q, w = systems.make(name)
    prec = "fp64" if w["prec"] == "fp64" else "fp32"
    plan, xd, qd, F, phi, Ed = setup_plan(se, torch, tuning, x, q, w, prec, tile=args.tile,
                                          variant=args.variant)
    total_ms, K, clk = time_steps(torch, lambda: plan.evaluate(xd, qd, F, phi, Ed), K, W, flush,
                                  ws=ws)
    if ws > 1:
        from paper_1712_04718_gb300.sharding import max_over_ranks
        total_ms = max_over_ranks(total_ms, ws, "cuda")
    p = plan.params()
    plan.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": ws * K / (total_ms / 1e3), "unit": "evals/s",
                          "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": total_ms / K,
                          "bare": True, "config": {"workload": name,
                                                   "spread_variant": int(p["spread_variant"]),
                                                   "spread_tile": int(p["tile"])},
                          "clocks": clk}))


# ---------------------------------------------------------------------------
# Extras (--extras FILE): legs beyond the metric, written to a file

def run_extras(args, se, torch, res, flush):
    """Evaluation modes, real space, xi balance, no-graph and unsorted
    variants, per-stage events and the cost model of the headline workload."""
    if "x" not in res:
        return {}
    x, q, w, prec = res["x"], res["q"], res["w"], res["prec"]
    K = min(res["K"], 500)
    cfg = res["plan_cfg"]
    out = {"workload": res["workload"]}
    plan = se.Plan(len(q), w["L"], w["xi"], w["M"], w["P"], precision=prec)
    if prec != "fp64":
        plan.set_tuning(*cfg)
    dt = plan.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    F = torch.empty((len(q), 3), dtype=dt, device="cuda")
    phi = torch.empty((len(q),), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.set_graph(False)
    ms, k, _ = time_steps(torch, lambda: plan.evaluate(xd, qd, F, phi, Ed), K, 5, flush)
    out["no_graph"] = {"value": k / (ms / 1e3), "ms_per_step": ms / k}
    plan.set_graph(True)
    plan.set_timing(True)
    for _ in range(200):
        flush()
        plan.evaluate(xd, qd, F, phi, Ed)
    torch.cuda.synchronize()
    plan.set_timing(False)
    stages, nstage = plan.get_timing(reset=True)
    out["stage_events_us"] = {k: v / max(1, nstage) * 1e3 for k, v in stages.items()}
    out["cost_model"] = cost_model(stages, nstage, len(q), w["M"], w["P"], cfg[0])
    if prec != "fp64" and w["M"] <= 128:
        p4 = se.Plan(len(q), w["L"], w["xi"], w["M"], w["P"], precision=prec, spread_variant=4)
        ms, k, _ = time_steps(torch, lambda: p4.evaluate(xd, qd, F, phi, Ed), K, 5, flush)
        out["unsorted_variant"] = {"value": k / (ms / 1e3), "ms_per_step": ms / k}
        p4.close()
    plan.close()
    out["modes"] = other_modes(se, torch, x, q, w, prec, K, flush, cfg, res["F"])
    out["real_space"] = real_space(se, torch, x, q, w, prec, K, flush, cfg)
    if prec != "fp64":
        out["xi_balance"] = xi_balance(se, torch, x, q, w, prec)
    return out


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


def other_modes(se, torch, x, q, w, prec, K, flush, cfg, F_analytic):
    """The workload in the evaluation modes beside the headline's: forces by
    ik differentiation (the cuFFT pipeline with three more inverse FFTs and a
    four-grid gather), potential only (the gather without force sums) and
    energy only (no gather).  Same timing as the headline; the ik forces'
    difference from the analytic ones is given beside them."""
    N = len(q)
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
        ms, k, _ = time_steps(torch, lambda: plan.evaluate(xd, qd, F, phi, Ed), K, 10, flush)
        r = {"value": k / (ms / 1e3), "ms_per_step": ms / k,
             "spread_variant": int(plan.params()["spread_variant"])}
        if F is not None:
            r["rel_diff_from_analytic"] = rel_rms(F.double().cpu().numpy(), F_analytic)
        out[mode] = r
        plan.close()
    return out


def real_space(se, torch, x, q, w, prec, K, flush, cfg):
    """The real-space part of the Ewald sum (cell lists, cut-off 1 nm, or L/3
    for boxes under 3 nm) on the same input, alone and after the k-space
    evaluation into the same outputs (the whole Ewald sum)."""
    N = len(q)
    rc = min(1.0, w["L"] / 3.0)
    rprec = "fp64" if prec == "fp64" else "fp32"
    rs = se.RealSpace(N, w["L"], w["xi"], rc, precision=rprec)
    plan = se.Plan(N, w["L"], w["xi"], w["M"], w["P"], precision=prec)
    if prec != "fp64":
        plan.set_tuning(*cfg)
    dt = rs.dtype
    xd = torch.tensor(x, dtype=dt, device="cuda")
    qd = torch.tensor(q, dtype=dt, device="cuda")
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty((N,), dtype=dt, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = {"rc": rc, "cells_per_dim": rs.cells_per_dim(), "precision": rprec}
    for key, both in (("real_only", False), ("whole_ewald", True)):
        def step():
            if both:
                plan.evaluate(xd, qd, F, phi, Ed)
            rs.evaluate(xd, qd, F, phi, Ed, accumulate=both)
        ms, k, _ = time_steps(torch, step, K, 10, flush)
        out[key] = {"value": k / (ms / 1e3), "ms_per_step": ms / k}
    rs.close()
    plan.close()
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


# ---------------------------------------------------------------------------
# Reference arm

def run_reference(args):
    """Reference arm: the FP64 CPU oracle (plain SE, O2) on the host cores,
    for the same workload, metric and unit."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    from paper_1712_04718_gb300 import systems
    if args.workload.startswith("ensemble"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm times single-system workloads only"}))
        return
    x, q, w = systems.make(args.workload)
    xd, qd = np.asarray(x, np.float64), np.asarray(q, np.float64)
    cm = 64 if w["prec"] == "fp64" else 32
    t0 = time.perf_counter()
    oracle.se_kspace(xd, qd, w["L"], w["xi"], w["M"], w["P"], cell_mode=cm)
    one = time.perf_counter() - t0
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
