#!/usr/bin/env python3
"""Throughput of the spectral Poisson solve -Δu = f (periodic, unit cube).

One step = one full solve (forward 3D FFT, division by 4π²|k|², inverse 3D
FFT) of the 512^3 FP32 sharp-source workload: one periodised Gaussian of
width 0.01 plus 4 smooth modes (|k| <= 4), mean removed, seeded.  Inputs and
outputs (512 MiB each) are larger than L2, so no flush is needed between
steps.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torchrun; the solve does not shard, so
every rank runs an independent replica (weak scaling, no collective on the
data path); value = units of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("unknowns/s & % HBM roofline at 512³; TC/batched vs plain FP32 at rel-L2 ≤1e-5")
UNIT = "unknowns/s"
WORKLOAD = "sharp_source 512^3: 1 periodised Gaussian sigma=0.01 + 4 modes |k|<=4, mean removed"
BYTES_PER_UNKNOWN_PER_PASS = 8  # FP32: each pass reads and writes the whole array once
PROFILE_EVERY = 8  # solves per profiled solve inside the timed region
E2E_STREAMS = 3  # host-buffer solves in flight (the library's staging ring holds three)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=512)
    ap.add_argument("--workload", choices=["sharp", "batch64"], default="sharp",
                    help="sharp: one FP32 grid^3 solve per step (default, 512^3); batch64: the 64 "
                         "uneven radix-2/3 grids in one persistent launch per step")
    ap.add_argument("--precision", choices=["f32", "f32_tc"], default="f32",
                    help="f32: FP32 butterflies; f32_tc: radix-16 stages of the y/x passes on the "
                         "tensor cores (FP16 hi/lo, row-scaled, FP32 accumulation)")
    ap.add_argument("--operator", choices=["poisson", "helmholtz", "fd"], default="poisson",
                    help="operator the solve inverts: -Δu = f (default), -Δu + c·u = f, or the "
                         "7-point finite-difference Laplacian; same passes, another multiplier")
    ap.add_argument("--helmholtz-c", type=float, default=1.0)
    ap.add_argument("--check", action="store_true",
                    help="also report this run's rel-L2 against the FP64 oracle (a few s of CPU; "
                         "batch64: worst and median over the 64 grids, batched and one plan per grid)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="--impl reference: OpenMP threads of the FP64 oracle (0: all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="default line: leave out the tensor-core and batched records (and their "
                         "oracle checks) that follow the FP32 timed region")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, values, device):
    """Element-wise maximum of `values` (floats) over all ranks; the values
    themselves when there is no process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_value(ws: int, units_per_rank: float, ms_per_step: float) -> float:
    """Whole-job throughput: every rank solves its own replica, so the job
    does ws times the units of one rank in the slowest rank's time."""
    return ws * units_per_rank / (ms_per_step * 1e-3)


def emit(line: dict, rank: int) -> bool:
    """Print the JSON line on rank 0 only; True if this rank printed."""
    if rank != 0:
        return False
    print(json.dumps(line), flush=True)
    return True


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clocks(out)


def parse_clocks(out: str) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi CSV rows of ClockSampler.FIELDS (no header, no units)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
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
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# Sources of the kernels whose DRAM traffic profiles/ncu_traffic.json records
# (the z bulk and TMA y/x passes): their translation units, every header they
# include, and the host code that picks their configurations and grids (the
# planner, the tuner and the pass pipeline).
TRAFFIC_SOURCES = ("paper_1408_6497_gb300/csrc/strided_tma.cu", "paper_1408_6497_gb300/csrc/zpass_bulk.cu",
                   "paper_1408_6497_gb300/csrc/launch.h", "paper_1408_6497_gb300/csrc/passes.cuh",
                   "paper_1408_6497_gb300/csrc/fft_core.cuh", "paper_1408_6497_gb300/csrc/tc.cuh",
                   "paper_1408_6497_gb300/csrc/tma.cuh", "paper_1408_6497_gb300/csrc/plan.h",
                   "paper_1408_6497_gb300/csrc/planner.cu", "paper_1408_6497_gb300/csrc/tuner.cu",
                   "paper_1408_6497_gb300/csrc/pipeline.cu", "include/psolve.h")


L2_BYTES = 129e6  # GB300 L2


def l2_note(shape) -> str:
    """How the timed solves relate to L2: every pass reads and writes the
    whole half spectrum (the z passes also f or u), with no flush between."""
    nx, ny, nz = shape
    real = 4 * nx * ny * nz
    spec = 8 * nx * ny * (nz // 2 + 1)
    sizes = f"f and u {real / 2**20:.0f} MiB each, spectrum {spec / 2**20:.0f} MiB"
    if spec > L2_BYTES:
        return f"every pass's arrays larger than the 129 MB L2 ({sizes}), no flush"
    return f"L2-influenced: the spectrum fits in the 129 MB L2 ({sizes}), no flush"


def solve_dram_frac(passes_ms: dict, unknowns: int, ms_per_step: float, peak: float,
                    shape=(512, 512, 512), operator: str = "poisson"):
    """Whole-solve DRAM rate as a fraction of the peak: the recorded ncu
    bytes of every pass of one solve over the event-timed solve; None if a
    pass has no record for the current sources."""
    total = 0.0
    for name in passes_ms:
        t = recorded_traffic(name, unknowns, shape, operator)
        if t is None:
            return None
        total += t
    return (total / (ms_per_step * 1e-3) / 1e9) / peak if passes_ms else None


_C_TOKENS = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'', re.S)


def code_only(text: str) -> str:
    """C/C++/CUDA source without its comments (string and character literals
    kept), so that comment edits do not count as kernel changes."""
    return _C_TOKENS.sub(lambda m: " " if m.group(0).startswith("/") else m.group(0), text)


def kernel_digest(read=None) -> str:
    """Hash of TRAFFIC_SOURCES without comments; `read(path)` returns a
    file's text (default: the working tree)."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(f.encode())
        h.update(code_only(text).encode())
    return h.hexdigest()[:16]


def recorded_traffic(pass_name: str, unknowns: int, shape=(512, 512, 512), operator: str = "poisson"):
    """DRAM bytes per launch of the pass's kernel from the committed ncu
    summary (profiles/ncu_traffic.json), only for the kernels it was taken
    on: the same grid (other grids run other line-length instantiations),
    the Poisson multiplier (other operators have their own x-pass
    instantiation) and the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p) or operator != "poisson":
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_digest") != kernel_digest() or list(d.get("grid", [])) != list(shape):
        return None
    e = d.get("passes", {}).get(pass_name)
    if not e:
        return None
    return float(e["dram_bytes_per_launch"]) * unknowns / float(e["unknowns"])


# --------------------------------------------------------------- oracle
def oracle_rate(grid: int, max_seconds: float, min_reps: int = 1):
    """Unknowns/s of the FP64 CPU oracle (as it stands) on the same source
    sampled on a grid^3 mesh; repeats until max_seconds is used."""
    import oracle
    from paper_1408_6497_gb300 import workloads as wl
    oracle.build()
    f = wl.sharp_source((grid,) * 3).f
    times = []
    t_all = time.perf_counter()
    while len(times) < min_reps or (time.perf_counter() - t_all) < max_seconds * 0.5:
        t0 = time.perf_counter()
        oracle.solve(f)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > max_seconds:
            break
    t = statistics.median(times)
    return grid ** 3 / t, t, len(times), oracle.threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1408_6497_gb300 import workloads as wl
    oracle.build()
    oracle.set_threads(args.oracle_threads)
    if args.workload == "batch64":
        return run_reference_batch(args, oracle, wl, ws, rank)
    # Size each step so that warmup + steps fit in about two minutes.
    probe_t = None
    grid = 64
    for g in (64, 128, 256, 512):
        f = wl.sharp_source((g,) * 3).f
        t0 = time.perf_counter()
        oracle.solve(f)
        dt = time.perf_counter() - t0
        if (args.steps + args.warmup) * dt > 120.0 and g > 64:
            break
        grid, probe_t = g, dt
        if g >= args.grid:
            break
    f = wl.sharp_source((grid,) * 3).f
    for _ in range(args.warmup):
        oracle.solve(f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(f)
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = grid ** 3 / (el / args.steps)
    sample = (f"{args.steps} FP64 oracle solves of the same source on a {grid}^3 grid "
              f"(each step bounded so the run ends within minutes)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("512^3", f"{grid}^3 sample of the 512^3 workload"),
                       "grid": [grid] * 3, "precision": "f64", "device": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, rank)
    return 0


def run_reference_batch(args, oracle, wl, ws, rank):
    """The oracle on the 64-grid batch: each step solves the first m grids,
    m as large as lets warmup + steps end within about two minutes."""
    shapes = wl.batch_shapes(64)
    fs = [wl.batch_instance(s, b).f for b, s in enumerate(shapes)]
    m = batch_sample_size(oracle, fs, 120.0 / max(1, args.steps + args.warmup))
    sample = fs[:m]
    n = sum(f.size for f in sample)
    for _ in range(args.warmup):
        for f in sample:
            oracle.solve(f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for f in sample:
            oracle.solve(f)
    el = time.perf_counter() - t0
    value = n / (el / args.steps)
    desc = (f"{args.steps} FP64 oracle solve(s) of the first {m} of the 64 uneven grids "
            f"({n} unknowns per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batch64: 64 uneven grids, axes from {24, ..., 256}, 16 Gaussians each"
                                   + ("" if m == len(fs) else f" (first {m} grids)"),
                       "grids": m, "precision": "f64", "device": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, rank)
    return 0


# ------------------------------------------------------------------ ours
def timed_solves(torch, plan, f, u, steps, dev, stream, barrier, profile=True):
    """K solves of `plan` timed with CUDA events on the launching stream,
    after a 2 s soak that brings the clocks to steady state; nvidia-smi
    samples the clocks over soak and timed region.  Returns (ms per solve,
    {pass: mean ms} over the profiled solves, clock record)."""
    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    soak_end = time.perf_counter() + 2.0
    while time.perf_counter() < soak_end:
        for _ in range(20):
            plan.execute(f, u)
        torch.cuda.synchronize(dev)
    # Per-pass events on every PROFILE_EVERY-th solve only: a recorded solve
    # runs its passes strictly back to back, the others overlap each pass's
    # set-up with the previous pass's drain.
    if profile:
        plan.set_profiling(PROFILE_EVERY)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.execute(f, u)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    avg = {}
    if profile:
        plan.set_profiling(False)
        pass_ms, nsol = plan.pass_times()
        avg = {k: v / max(1, nsol) for k, v in pass_ms.items()}
    return e0.elapsed_time(e1) / steps, avg, clocks


def tc_record(torch, args, f, f_np, N, shape, dev, stream, barrier, peak, ref):
    """The tensor-core form of the same solve (radix-16 stages of the y and x
    passes on tcgen05, FP16 hi/lo operands), timed like the FP32 line, with
    its rel-L2 and rel-ℓ∞ against the FP64 oracle."""
    from paper_1408_6497_gb300 import Plan
    plan = Plan(shape, dtype="f32_tc", device=dev)
    if not args.no_autotune:
        plan.autotune()
    u = torch.empty_like(f)
    for _ in range(max(3, args.warmup)):
        plan.execute(f, u)
    torch.cuda.synchronize(dev)
    ms, avg, clocks = timed_solves(torch, plan, f, u, args.steps, dev, stream, barrier)
    rec = {"precision": "f32_tc", "dtype": "f32+fp16x3-tc", "ms_per_step": ms, "value": N / (ms * 1e-3),
           "unit": UNIT, "passes_ms": {k: round(v, 5) for k, v in avg.items()},
           "solve_dram_frac": solve_dram_frac(avg, N, ms, peak, shape),
           "min_traffic_frac": (8 * N / (ms * 1e-3) / 1e9) / peak,
           "gpu_launches": plan.launches_per_solve * args.steps, "clocks": clocks}
    if ref is not None:
        plan.execute(f, u)
        ut = u.cpu().numpy().reshape(shape)
        import oracle
        rec["rel_l2_vs_oracle"] = oracle.rel_l2(ut, ref)
        rec["rel_linf_vs_oracle"] = oracle.rel_linf(ut, ref)
    plan.close()
    return rec


def batch64_record(torch, args, dev, stream, barrier, peak, check):
    """The 64 uneven radix-2/3 grids in one persistent launch per step (one
    graph replay), timed like the FP32 line; worst and median rel-L2 of the
    64 solutions against the FP64 oracle."""
    from paper_1408_6497_gb300 import Plan
    from paper_1408_6497_gb300 import workloads as wl
    shapes = wl.batch_shapes(64)
    N = sum(int(np.prod(s)) for s in shapes)
    plan = Plan(dtype="f32", shapes=shapes, device=dev)
    if not args.no_autotune:
        plan.autotune()
    flat = plan.empty()
    fs = []
    for b, s in enumerate(shapes):
        fb = wl.batch_instance(s, b).f.astype(np.float32)
        fs.append(fb)
        plan.view(flat, b).copy_(torch.from_numpy(fb))
    u = torch.empty_like(flat)
    for _ in range(max(3, args.warmup)):
        plan.execute(flat, u)
    torch.cuda.synchronize(dev)
    ms, _, clocks = timed_solves(torch, plan, flat, u, args.steps, dev, stream, barrier, profile=False)
    algo = 5 * BYTES_PER_UNKNOWN_PER_PASS * N
    rec = {"workload": "64 FP32 grids, axes drawn from {24,32,48,64,96,128,192,256}, 16 periodised "
                       "Gaussians each, one persistent launch per step", "unknowns": N,
           "ms_per_step": ms, "value": N / (ms * 1e-3), "unit": UNIT,
           "solve_dram_frac": (algo / (ms * 1e-3) / 1e9) / peak,
           "solve_dram_frac_basis": "algorithmic bytes (5 passes x 8 B per unknown) over the event time",
           "gpu_launches": plan.launches_per_solve * args.steps, "clocks": clocks}
    if check:
        import oracle
        plan.execute(flat, u)
        errs = batch_errors(oracle, fs, [plan.view(u, b).cpu().numpy() for b in range(64)])
        rec["rel_l2_vs_oracle"] = {"worst": max(errs), "median": statistics.median(errs)}
    plan.close()
    return rec


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"impl": "ours", "error": "no CUDA device"}))
        return 1
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1408_6497_gb300 import Plan, build
    from paper_1408_6497_gb300 import workloads as wl
    build.build()

    n = args.grid
    shape = (n, n, n)
    N = n ** 3
    f_np = wl.sharp_source(shape).f.astype(np.float32)
    f_host = torch.from_numpy(f_np.ravel())
    f_pin = f_host.pin_memory()
    u_pin = torch.empty_like(f_pin).pin_memory()
    f = f_pin.to(dev)
    u = torch.empty_like(f)
    plan = Plan(shape, dtype=args.precision, device=dev, operator=args.operator, c=args.helmholtz_c)
    if not args.no_autotune:
        plan.autotune()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        plan.execute(f, u)
    torch.cuda.synchronize(dev)

    ms_step, avg, clocks = timed_solves(torch, plan, f, u, args.steps, dev, stream, barrier)

    # End to end through the public host-buffer API: every step reads its f
    # from pinned host memory and writes its u back to pinned host memory.
    # Steps rotate over E2E_STREAMS streams and buffer pairs, so one step's
    # output traffic overlaps the next step's input traffic on the host link
    # while another step computes.
    e2e_steps = max(6, min(args.steps, 12))
    NS = E2E_STREAMS
    f_pins = [f_pin] + [f_host.clone().pin_memory() for _ in range(NS - 1)]
    u_pins = [u_pin] + [torch.empty_like(f_pin).pin_memory() for _ in range(NS - 1)]
    streams = [torch.cuda.Stream(dev) for _ in range(NS)]
    for k in range(2 * NS):
        plan.execute_host_async(f_pins[k % NS], u_pins[k % NS], streams[k % NS])
    torch.cuda.synchronize(dev)
    barrier()
    # three timed runs of e2e_steps steps each; the median run is reported
    # (the host link is shared with the machine's other GPUs' traffic)
    runs = []
    for _ in range(3):
        h0 = time.perf_counter()
        for k in range(e2e_steps):
            plan.execute_host_async(f_pins[k % NS], u_pins[k % NS], streams[k % NS])
        torch.cuda.synchronize(dev)
        runs.append((time.perf_counter() - h0) / e2e_steps)
    e2e_s = sorted(runs)[1]
    # the synchronous call, one step at a time, for reference
    plan.execute_host(f_pin, u_pin)
    h1 = time.perf_counter()
    for _ in range(3):
        plan.execute_host(f_pin, u_pin)
    e2e_sync_s = (time.perf_counter() - h1) / 3
    barrier()

    el_ms, e2e_s, e2e_sync_s = max_over_ranks(dist, [ms_step * args.steps, e2e_s, e2e_sync_s], dev)

    ms_per_step = el_ms / args.steps
    value = job_value(ws, N, ms_per_step)
    top = max(avg, key=avg.get)
    peak, peak_kind = peaks()
    algo_bytes = BYTES_PER_UNKNOWN_PER_PASS * N
    achieved = algo_bytes / (avg[top] * 1e-3) / 1e9
    traffic = recorded_traffic(top, N, shape, args.operator)

    # The comparison the metric asks for: the tensor-core and batched forms
    # next to this plain FP32 single solve, each with its error against the
    # FP64 oracle (the default line only; one GPU).
    compare = (ws == 1 and args.precision == "f32" and args.operator == "poisson" and n == 512
               and not args.no_compare)
    check = args.check or compare
    ref = None
    if check and rank == 0:
        import oracle
        oracle.build()
        ref = oracle.solve(f_np.astype(np.float64), op=args.operator, c=args.helmholtz_c)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    line = {
        "impl": "ours", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "f32" else "f32+fp16x3-tc",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("512^3", f"{shape[0]}^3"), "grid": list(shape),
                   "precision": args.precision,
                   "operator": args.operator + (f" c={args.helmholtz_c}" if args.operator == "helmholtz" else ""),
                   "l2": l2_note(shape),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "clock_window": "2 s soak + timed region"},
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "algorithmic_bytes_per_launch": algo_bytes},
        "passes_ms": {k: round(v, 5) for k, v in avg.items()},
        "min_traffic_frac": (8 * N / (ms_per_step * 1e-3) / 1e9) / peak,
        "solve_dram_frac": solve_dram_frac(avg, N, ms_per_step, peak, shape, args.operator),
        "e2e": {"value": ws * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * N, "api": f"psolve_execute_host_async, pinned buffers, {NS} streams",
                "runs_ms": [round(r * 1e3, 4) for r in runs], "sync_call_value": ws * N / e2e_sync_s},
        "gpu_launches": plan.launches_per_solve * args.steps,
        "clocks": clocks,
    }
    if ref is not None:
        import oracle
        plan.execute(f, u)
        uh = u.cpu().numpy().reshape(shape)
        line["rel_l2_vs_oracle"] = oracle.rel_l2(uh, ref)
        line["rel_linf_vs_oracle"] = oracle.rel_linf(uh, ref)
    if compare:
        plan.close()
        line["tc"] = tc_record(torch, args, f, f_np, N, shape, dev, stream, barrier, peak, ref)
        line["tc"]["vs_fp32_single_solve"] = line["tc"]["value"] / value
        line["batch64"] = batch64_record(torch, args, dev, stream, barrier, peak, True)
        line["batch64"]["vs_fp32_single_solve"] = line["batch64"]["value"] / value
    if ws == 1 and not args.no_cpu_baseline:
        rate, t, reps, cores = oracle_rate(min(n, 256), max_seconds=20.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{reps} FP64 oracle solve(s) of the same source on a "
                                          f"{min(n, 256)}^3 grid, median {t:.2f} s"}
    emit(line, rank)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ batch of 64
def batch_sample_size(oracle, fs, budget_s: float) -> int:
    """How many leading grids of `fs` one oracle pass solves within about
    `budget_s` seconds (at least one), from the time of the first."""
    t0 = time.perf_counter()
    oracle.solve(fs[0])
    per_unknown = (time.perf_counter() - t0) / fs[0].size
    m, n = 0, 0
    while m < len(fs) and (m == 0 or (n + fs[m].size) * per_unknown <= budget_s):
        n += fs[m].size
        m += 1
    return m


def batch_errors(oracle, fs, us):
    """rel-L2 of each instance's solution `us[b]` against the FP64 oracle
    solve of the same (FP32-rounded) right-hand side `fs[b]`."""
    return [oracle.rel_l2(u, oracle.solve(np.asarray(f, dtype=np.float64))) for f, u in zip(fs, us)]


def run_batch(args):
    """64 uneven grids (axes from {24..256}) per step in one persistent launch,
    next to the same 64 solves issued one plan per instance (the plain FP32
    single-solve path)."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1408_6497_gb300 import Plan, build
    from paper_1408_6497_gb300 import workloads as wl
    build.build()
    shapes = wl.batch_shapes(64)
    N = sum(int(np.prod(s)) for s in shapes)
    plan = Plan(dtype="f32", shapes=shapes, device=dev)
    if not args.no_autotune:
        plan.autotune()
    flat = plan.empty()
    for b, s in enumerate(shapes):
        plan.view(flat, b).copy_(torch.from_numpy(wl.batch_instance(s, b).f.astype(np.float32)))
    u = torch.empty_like(flat)
    singles = [Plan(s, dtype="f32", device=dev) for s in shapes]
    if not args.no_autotune:
        for sp in singles:
            sp.autotune()
    views_f = [plan.view(flat, b).reshape(-1) for b in range(64)]
    views_u = [plan.view(u, b).reshape(-1) for b in range(64)]
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        plan.execute(flat, u)
        for b, sp in enumerate(singles):
            sp.execute(views_f[b], views_u[b])
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(args.steps):
        plan.execute(flat, u)
    e1.record(stream)
    for _ in range(args.steps):
        for b, sp in enumerate(singles):
            sp.execute(views_f[b], views_u[b])
    e2.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    t_batch = e0.elapsed_time(e1) / args.steps
    t_single = e1.elapsed_time(e2) / args.steps
    peak, peak_kind = peaks()
    algo = 5 * BYTES_PER_UNKNOWN_PER_PASS * N
    achieved = algo / (t_batch * 1e-3) / 1e9
    h_pin = flat.cpu().pin_memory()
    o_pin = torch.empty_like(h_pin).pin_memory()
    plan.execute_host(h_pin, o_pin)
    h0 = time.perf_counter()
    for _ in range(5):
        plan.execute_host(h_pin, o_pin)
    e2e_s = (time.perf_counter() - h0) / 5
    line = {
        "impl": "ours", "metric": METRIC, "value": N / (t_batch * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64: 64 FP32 grids, axes drawn from {24,32,48,64,96,128,192,256}, "
                               "16 periodised Gaussians each, one persistent launch per step",
                   "unknowns": N, "l2": "working set 255 MiB > L2, no flush"},
        "roofline": {"bound": "hbm", "kernel": "batched", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": algo},
        "single_solve_loop": {"value": N / (t_single * 1e-3), "ms_per_step": t_single,
                              "launches_per_step": sum(sp.launches_per_solve for sp in singles)},
        "batched_vs_single_solve_loop": t_single / t_batch,
        "e2e": {"value": N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * plan.total,
                "d2h_bytes_per_step": 4 * plan.total},
        "gpu_launches": plan.launches_per_solve * args.steps,
        "clocks": clocks,
    }
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        fs64 = [wl.batch_instance(s, b).f for b, s in enumerate(shapes)]
        m = batch_sample_size(oracle, fs64, 15.0)
        t0 = time.perf_counter()
        for f in fs64[:m]:
            oracle.solve(f)
        el = time.perf_counter() - t0
        n = sum(f.size for f in fs64[:m])
        line["cpu_baseline"] = {"value": n / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                                "sample": f"FP64 oracle solves of the first {m} of the 64 grids "
                                          f"({n} unknowns, {el:.1f} s)"}
    if args.check and rank == 0:
        import oracle
        oracle.build()
        u2 = torch.empty_like(flat)
        plan.execute(flat, u)
        for b, sp in enumerate(singles):
            sp.execute(views_f[b], plan.view(u2, b).reshape(-1))
        torch.cuda.synchronize(dev)
        fs = [plan.view(flat, b).cpu().numpy() for b in range(64)]
        for key, out in (("rel_l2_vs_oracle", u), ("single_solve_loop_rel_l2_vs_oracle", u2)):
            errs = batch_errors(oracle, fs, [plan.view(out, b).cpu().numpy() for b in range(64)])
            line[key] = {"worst": max(errs), "median": statistics.median(errs)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
