#!/usr/bin/env python
"""Benchmark: the five-kernel convolution sweep on batches of 16 seeded densities (Sec. 2.1,
eq. (An)), on one GB300 per rank.

One step = the batch of 16 densities (sums of 1-8 C-infinity bumps, n x n, b = 3) convolved with
each of log|x|, |x|^-1/2, |x|^-1, |x|^-3/2 and (i/4) H0(20 |x|): 80 convolutions.  The headline is
the FP64 path (the paper's arithmetic) at n = 4096; the FP32 path, n = 2048 and 8192, the
Lippmann-Schwinger solver and the serving loop are reported beside it, and every timed sweep
carries its error against the FP64 oracle for density 0 of each kernel (computed after the timed
region).  Inputs (16 x 4096^2 x 8 B = 2.1 GB) exceed the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp32]
"""
import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 and FP64 FMA rates of the GPU from its unit counts and clock (context beside the measured
# microbenchmark peaks the rooflines divide by): 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz, and
# GB300's nominal 1.25 TFLOP/s FP64.
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_NOMINAL_TFLOPS = 1.25

METRIC = ("convolutions/s & HBM-roofline % at N=2048²/4096² (FP64 vs mixed); "
          "LS solves/s, p99 latency")
SWEEP = [("log", {"scale": 1.0}), ("pow", {"gamma": -0.5}), ("pow", {"gamma": -1.0}),
         ("pow", {"gamma": -1.5}), ("helmholtz", {"kappa": 20.0})]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--no-extras", action="store_true", help="headline only (no FP64/n=2048/LS legs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the error of the timed outputs against the oracle")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                    help="arithmetic of the headline sweep (the other is reported beside it)")
    ap.add_argument("--only", choices=["r2r", "r2r64", "r2c", "r2c64", "c2c"], default=None,
                    help="profiling case: warmup + steps applies of one plan (log kernel R2R FP32, "
                         "R2R FP64, Helmholtz R2C FP32 or FP64, C2C FP32), no other legs")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "mine" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value, device="cuda"):
    """Slowest rank's time (the job's time for replicas that run concurrently)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, units_per_rank, ms_max):
    """Whole-job rate of N replicas: all ranks' units over the slowest rank's time."""
    return ws * units_per_rank / (ms_max * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = ["-i", str(device_index)]
        self.cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                    "-lms", "200"] + sel

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- traffic record
# The files the pass kernels and their launches are built from: kernels, transforms and copies
# (*.cuh), shared declarations (*.h), the launch configuration and instantiations (passes*.cu),
# the multiplier tables (ghat.cu), the plan's sizes (plan.cu) and the TMA maps (tma.cu).  The
# LS solver, serving runtime, host-buffer pipeline, graph groups, masks and peak probes are not.
KERNEL_SOURCES = ("*.cuh", "*.h", "passes*.cu", "ghat.cu", "plan.cu", "tma.cu")


def kernel_source_hash():
    csrc = os.path.join(ROOT, "paper_2107_03958_gb300", "csrc")
    files = sorted(set(f for pat in KERNEL_SOURCES for f in glob.glob(os.path.join(csrc, pat))))
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(name):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current kernel
    sources (the summary records the hash of csrc/); else None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(rec["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- measured peaks
def peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def hbm_peak():
    p = peaks_file()
    for k in ("hbm_gbs", "copy_gbs", "hbm_copy_gbs"):
        if k in p:
            return float(p[k]), "measured (MEASURED_PEAKS.json)"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle baseline
def cpu_oracle_rate(n, reps=1):
    """The oracle's full FFT convolution (eq. (An)) of one density with log|x|, FP64, all host
    threads; returns (conv/s, threads, seconds)."""
    import oracle as O
    from paper_2107_03958_gb300 import inputs
    O.set_threads(os.cpu_count() or 1)
    threads = O.threads()
    M = 3 * n
    g = O.ghat_full("log", M, 3.0, O.default_trunc_radius(3.0), scale=1.0)
    u = inputs.bump_sums(n, 1)[0]
    t0 = time.perf_counter()
    for _ in range(reps):
        O.conv(u, M, g)
    dt = time.perf_counter() - t0
    return reps / dt, threads, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle as O
    from paper_2107_03958_gb300 import inputs
    n = args.n
    O.set_threads(os.cpu_count() or 1)
    M = 3 * n
    g = O.ghat_full("log", M, 3.0, O.default_trunc_radius(3.0), scale=1.0)
    us = inputs.bump_sums(n, args.batch)
    for w in range(args.warmup):
        O.conv(us[w % args.batch], M, g)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.conv(us[k % args.batch], M, g)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    sample = "one density of the batch per step (log kernel, n=%d, b=3, FP64 C oracle)" % n
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "conv/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": "conv/s", "cores": O.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "conv/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def workload_config(args):
    other = "fp32" if args.precision == "fp64" else "fp64"
    return {"workload": "kernel sweep batched: 16 seeded bump-sum densities x {log, |x|^-0.5, "
                        "|x|^-1, |x|^-1.5, Helmholtz kappa=20}, n=%d, b=3" % args.n,
            "n": args.n, "period_b": 3, "batch": args.batch, "kernels": 5,
            "convolutions_per_step": 5 * args.batch,
            "precision": "%s (headline), %s reported beside it" % (args.precision, other),
            "embedding": "compact: weights of eq. (quad_wts) from the period-3 moments, 2n-periodic "
                         "transforms (period-3 transforms reported as fp32_period_b)",
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas"}


# ---------------------------------------------------------------- GPU legs
def make_plans(n, batch, precision, compact, period=3):
    from paper_2107_03958_gb300.api import ConvPlan
    plans = []
    for kern, kw in SWEEP:
        io = "r2c" if kern == "helmholtz" else "r2r"
        plans.append(ConvPlan(kern, n=n, period=period, precision=precision, io=io, batch_max=batch,
                              compact=compact, **kw))
    return plans


def sweep_leg(n, batch, precision, steps, warmup, stream, timing=False, compact=True, period=3):
    """Time `steps` sweeps on device-resident inputs; returns dict with ms/step and the pass
    timings of the plans."""
    import torch
    from paper_2107_03958_gb300 import inputs
    plans = make_plans(n, batch, precision, compact, period)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.from_numpy(inputs.bump_sums(n, batch)).to(dt).cuda()
    outs = [torch.empty((batch, n, n), dtype=p.out_dtype(), device="cuda") for p in plans]

    def step():
        for p, o in zip(plans, outs):
            p.apply(u, out=o, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    if timing:
        for p in plans:
            p.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # density 0 of the last timed step, per kernel (for the error against the oracle)
    res = {"ms": ms, "plans": plans, "launches": 3 * len(plans) * steps,
           "out0": [o[0].cpu().numpy() for o in outs], "u0": u[0].double().cpu().numpy()}
    if timing:
        res["passes"] = [p.timing_read() for p in plans]
        for p in plans:
            p.timing(False)
    return res


def shared_rows_leg(n, batch, precision, steps, warmup, stream, compact=True):
    """The same sweep through conv_apply_multi: the five kernels' row transforms of pass 1 run
    once per step (they depend only on the densities), then passes 2 and 3 of each plan.  Each
    output is bitwise the independent apply's; reported beside the headline, which runs five
    independent applies."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import apply_multi, multi_workspace_bytes
    plans = make_plans(n, batch, precision, compact)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.from_numpy(inputs.bump_sums(n, batch)).to(dt).cuda()
    outs = [torch.empty((batch, n, n), dtype=p.out_dtype(), device="cuda") for p in plans]
    ws = torch.empty(multi_workspace_bytes(plans, batch), dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            apply_multi(plans, u, outs=outs, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            apply_multi(plans, u, outs=outs, workspace=ws, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    for p in plans:
        p.device_status()
    return {"value": 5 * batch / (ms * 1e-3), "unit": "conv/s", "ms_per_step": ms, "steps": steps,
            "launches_per_step": 1 + 2 * len(plans), "api": "conv_apply_multi"}


def e2e_leg(n, batch, steps, warmup, compact=True, precision="fp64"):
    """End to end through conv_apply_host_multi (the call that takes HOST buffers): every step
    uploads the batch of densities from pinned host memory once, runs the five plans' passes on
    each chunk and downloads every result into pinned host memory, each plan's result chunk
    behind the next plan's passes.  Timed with CUDA events from before the first upload to after
    the last download."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import apply_host_multi
    plans = make_plans(n, batch, precision, compact)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u_host = torch.from_numpy(inputs.bump_sums(n, batch)).to(dt).pin_memory()
    outs = [torch.empty((batch, n, n), dtype=p.out_dtype()).pin_memory() for p in plans]
    main = torch.cuda.current_stream()

    def step():
        apply_host_multi(plans, u_host, outs=outs, stream=main)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for _ in range(steps):
        step()
    e1.record(main)
    torch.cuda.synchronize()
    for p in plans:
        p.device_status()
    chunk = max(1, (batch + 3) // 4)
    return {"ms": e0.elapsed_time(e1), "launches": 3 * len(plans) * ((batch + chunk - 1) // chunk) * steps,
            "h2d": u_host.numel() * u_host.element_size(),
            "d2h": sum(o.numel() * o.element_size() for o in outs)}


def r2r_bytes(plan, batch):
    """Algorithmic HBM bytes of one column-pass launch (R2R): read and write the n x (L/2+1)
    spectra of the batch (L the transform length), read the multiplier quadrant once."""
    n, L = plan.n, plan.info.transform_len
    h = L // 2 + 1
    esz = 16 if plan.precision == "fp64" else 8
    return batch * 2 * h * n * esz + h * h * (esz // 2)


def oracle_reference(u0, n):
    """The FP64 oracle's A_n u0 (eq. (An), full period-3 grid) for each kernel of the sweep."""
    import oracle as O
    O.set_threads(os.cpu_count() or 1)
    M = 3 * n
    a = O.default_trunc_radius(3.0)
    refs = []
    for kern, kw in SWEEP:
        kind = "helm" if kern == "helmholtz" else kern
        g = O.ghat_full(kind, M, 3.0, a, **kw)
        r = O.conv(u0, M, g)
        refs.append(r if kern == "helmholtz" else r.real)
        del g
    return refs


def errors_vs_oracle(out0, refs):
    """Relative L-infinity error (eq. (rel-err)) of density 0 of each kernel against the oracle."""
    import numpy as np
    errs = {}
    for (kern, kw), o, r in zip(SWEEP, out0, refs):
        name = kern if kern != "pow" else "pow%g" % kw["gamma"]
        errs[name] = float(np.max(np.abs(o - r)) / np.max(np.abs(r)))
    return errs


def cols_roofline(run, batch, peak_tflops, hbm, peak_source):
    """Column-pass rooflines of the R2R plans of a timed sweep: the ALU view (5 L log2 L flops per
    transform, two transforms per column, h = L/2 + 1 columns per density) and the HBM view
    (algorithmic bytes of r2r_bytes)."""
    r = [(p, t) for p, t in zip(run["plans"], run["passes"]) if p.io == "r2r"]
    ms = sum(t[0][1] for _, t in r) / sum(t[1] for _, t in r)
    plan = r[0][0]
    L = plan.info.transform_len
    flops = 5.0 * L * math.log2(L) * 2 * (L // 2 + 1) * batch
    byts = r2r_bytes(plan, batch)
    tf = flops / (ms * 1e-3) / 1e12
    gbs = byts / (ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": tf, "peak": peak_tflops, "unit": "TFLOP/s", "frac": tf / peak_tflops,
            "peak_source": peak_source, "avg_launch_ms": ms, "transform_len": L,
            "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}}


def sweep_roofline(run, batch, prec, alu_peak, alu_nominal, hbm, hbm_src):
    """Roofline of a timed sweep's dominant kernel, the R2R column pass (forward column transform,
    multiplier, inverse column transform): bound by the SMs' FFT arithmetic in both precisions (its
    DRAM bytes equal the algorithmic bytes, at a fraction of the copy peak), so reported against
    the measured FMA rate of the same precision, with the HBM view beside it."""
    r2r = [(p, t) for p, t in zip(run["plans"], run["passes"]) if p.io == "r2r"]
    tot = [0.0, 0.0, 0.0]
    cnt = 0
    for p, (passes, applies) in r2r:
        for i in range(3):
            tot[i] += passes[i]
        cnt += applies
    col_ms = tot[1] / cnt
    plan = r2r[0][0]
    col_bytes = r2r_bytes(plan, batch)
    gbs = col_bytes / (col_ms * 1e-3) / 1e9
    L = plan.info.transform_len
    col_flops = (L // 2 + 1) * batch * 2 * 5.0 * L * math.log2(L)
    tf = col_flops / (col_ms * 1e-3) / 1e12
    tname = "double" if prec == "fp64" else "float"
    share = [t / sum(tot) for t in tot]
    return {"bound": "alu", "kernel": "kf_r2r_cols<%s> (column pass, compact embedding, L = 2n = %d)" % (tname, L),
            "achieved": tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": tf / alu_peak,
            "peak_source": "measured %s FMA microbenchmark (conv_measure_peaks, this run)" % prec.upper(),
            "peak_nominal": alu_nominal, "frac_of_nominal": tf / alu_nominal,
            "flops_model": "5 L log2 L per complex length-L transform, forward and inverse per column, "
                           "L/2+1 columns per density (the conventional count; the pruned first and "
                           "last stages do less)",
            "flops_per_launch": col_flops, "avg_launch_ms": col_ms,
            "traffic": recorded_traffic("kf_r2r_cols_%s_compact_n%d.txt" % (prec, plan.n)),
            "algorithmic_bytes_per_launch": col_bytes,
            "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_source": hbm_src},
            "pass_share_r2r": {"rows_fwd": share[0], "cols": share[1], "rows_inv": share[2]}}


def period3_view(n, batch, prec, col_ms, step_ms, hbm):
    """Effective bandwidth against the bytes the plain three-pass schedule on the period-3 grid
    (M = 3n, spectra of n x (3n/2 + 1) per density, multiplier quadrant (3n/2 + 1)^2) moves: per
    R2R convolution 65 n^2 B in FP32 (130 n^2 in FP64), per Helmholtz one 102 n^2 (204 n^2); the
    R2R column pass 24 n^2 per density + 9 n^2 per launch in FP32 (twice that in FP64).  The compact
    embedding moves fewer bytes than this, so these fractions credit it with the bytes it saves."""
    f = 2 if prec == "fp64" else 1
    nn = float(n) * n
    col = f * (24 * nn * batch + 9 * nn)
    step = f * batch * (4 * 65 * nn + 102 * nn)
    return {"model": "period-3 three-pass schedule bytes (FP32 65 n^2 per R2R conv, 102 n^2 per "
                     "Helmholtz conv; FP64 twice)",
            "col_bytes_per_launch": col, "col_gbs": col / (col_ms * 1e-3) / 1e9,
            "col_frac": col / (col_ms * 1e-3) / 1e9 / hbm,
            "step_bytes": step, "step_gbs": step / (step_ms * 1e-3) / 1e9,
            "step_frac": step / (step_ms * 1e-3) / 1e9 / hbm}


def n8192_leg(steps, stream, hbm, fp32_peak):
    """The largest grid of the discontinuous-density sweep: n = 8192, batch 8, log kernel, FP32 R2R
    on the compact grid (L = 16384, compile-time stages, 1024 threads per line)."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import ConvPlan
    n, B = 8192, 8
    t0 = time.perf_counter()
    plan = ConvPlan("log", n=n, period=3, precision="fp32", io="r2r", batch_max=B, compact=True)
    plan_s = time.perf_counter() - t0
    u = torch.from_numpy(inputs.bump_sums(n, B, seed=81)).float().cuda()
    out = torch.empty_like(u)
    with torch.cuda.stream(stream):
        for _ in range(2):
            plan.apply(u, out=out, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.apply(u, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan.timing(True)
    for _ in range(2):
        plan.apply(u, out=out, stream=stream)
    t, cnt = plan.timing_read()
    plan.timing(False)
    plan.device_status()
    col_ms = t[1] / cnt
    L = plan.info.transform_len
    flops = 5.0 * L * math.log2(L) * 2 * (L // 2 + 1) * B
    byts = r2r_bytes(plan, B)
    return {"value": B / (ms * 1e-3), "unit": "conv/s", "batch": B, "ms_per_batch": ms, "transform_len": L,
            "plan_build_s": plan_s, "pass_ms": [x / cnt for x in t],
            "roofline_cols": {"bound": "alu", "achieved": flops / (col_ms * 1e-3) / 1e12, "peak": fp32_peak,
                              "unit": "TFLOP/s", "frac": flops / (col_ms * 1e-3) / 1e12 / fp32_peak,
                              "peak_source": "measured FP32 FMA microbenchmark (conv_measure_peaks)",
                              "hbm": {"achieved": byts / (col_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                      "frac": byts / (col_ms * 1e-3) / 1e9 / hbm}}}


def ls_leg(n, kappa, repeats, stream):
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import ConvPlan, ls_solve
    m = torch.tensor(inputs.lippmann_contrast(n, "bump"), device="cuda")
    f = torch.tensor(inputs.plane_wave(n, kappa), device="cuda")
    out = {}
    for mode in ("fp64", "mixed"):
        plan = ConvPlan("helmholtz", n=n, period=3, precision="fp64" if mode == "fp64" else "fp32",
                        io="c2c", kappa=kappa, compact=True)
        ls_solve(plan, m, f, refine=(mode == "mixed"), stream=stream)  # warm-up
        lat, info = [], None
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = ls_solve(plan, m, f, refine=(mode == "mixed"), stream=stream)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0)
        lat.sort()
        out[mode] = {"solves_per_s": len(lat) / sum(lat), "p50_ms": 1e3 * lat[len(lat) // 2],
                     "p99_ms": 1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                     "iters": info["iters"], "rel_residual": info["rel_residual"]}
    return {"n": n, "kappa": kappa, "contrast": "0.5 bump(0.4)", "tol": 1e-10, "restart": 50,
            "repeats": repeats, **out}


def group_leg(reps, stream):
    """Mixed-size batching: the serving mix's grid sizes (n = 128 ... 2048, counts falling with n as
    the mix's weights do, the sweep's five kernels in turn, FP32 compact plans) applied once per
    step, either one conv_apply per size on one stream or as one ConvGroup graph launch."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import ConvGroup, ConvPlan
    sizes = [(128, 16), (256, 16), (512, 8), (1024, 4), (2048, 1)]
    items = []
    for i, (n, b) in enumerate(sizes):
        kern, kw = SWEEP[i % len(SWEEP)]
        io = "r2c" if kern == "helmholtz" else "r2r"
        p = ConvPlan(kern, n=n, period=3, precision="fp32", io=io, batch_max=b, compact=True, **kw)
        u = torch.from_numpy(inputs.bump_sums(n, b, seed=900 + i)).float().cuda()
        items.append((p, u, torch.empty((b, n, n), dtype=p.out_dtype(), device="cuda")))
    g = ConvGroup(items)
    convs = sum(b for _, b in sizes)

    def seq():
        for p, u, o in items:
            p.apply(u, out=o, stream=stream)

    def grp():
        g.launch(stream)

    out = {}
    for name, fn in (("sequential", seq), ("group", grp)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"conv_per_s": convs / (ms * 1e-3), "ms_per_step": ms}
    for p, _, _ in items:
        p.device_status()
    return {"sizes_batches": sizes, "convolutions_per_step": convs, "reps": reps,
            "launches_per_step": {"sequential": 3 * len(sizes), "group": "1 graph of %d kernels" % (3 * len(sizes))},
            "working_set": "about 0.2 GB of inputs, outputs and spectra, partly L2-resident", **out,
            "speedup": out["sequential"]["ms_per_step"] / out["group"]["ms_per_step"]}


def ls_multi_leg(n, kappa, K, repeats, stream):
    """K incident directions (angles 2 pi s / K) on the bump scatterer: one stacked solve
    (ls_solve_multi, batched matvecs) against K single solves, both to 1e-10 per system."""
    import numpy as np
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import ConvPlan, ls_solve, ls_solve_multi
    m = torch.tensor(inputs.lippmann_contrast(n, "bump"), device="cuda")
    F = torch.tensor(np.stack([inputs.plane_wave(n, kappa, 2 * math.pi * s / K) for s in range(K)]), device="cuda")
    out = {"n": n, "kappa": kappa, "rhs": K, "tol": 1e-10, "repeats": repeats}
    for mode in ("mixed", "fp64"):
        plan = ConvPlan("helmholtz", n=n, period=3, precision="fp64" if mode == "fp64" else "fp32",
                        io="c2c", kappa=kappa, compact=True)
        refine = mode == "mixed"

        def single():
            return [ls_solve(plan, m, F[s], refine=refine, stream=stream)[1] for s in range(K)]

        def multi():
            return ls_solve_multi(plan, m, F, refine=refine, stream=stream)[1]

        res = {}
        for name, fn in (("single", single), ("stacked", multi)):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(repeats):
                infos = fn()
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) / repeats
            res[name] = {"solves_per_s": K / wall, "ms_per_batch": 1e3 * wall,
                         "iters": [i["iters"] for i in infos][:1] if name == "stacked" else [i["iters"] for i in infos],
                         "max_rel_residual": max(i["rel_residual"] for i in infos)}
        res["speedup"] = res["single"]["ms_per_batch"] / res["stacked"]["ms_per_batch"]
        out[mode] = res
        del plan
        torch.cuda.empty_cache()
    return out


def profile_case(args):
    """Small fixed case for ncu captures: one plan, warmup + steps applies, nothing else."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import ConvPlan
    prec = "fp64" if args.only in ("r2r64", "r2c64") else "fp32"
    compact = os.environ.get("BENCH_PERIOD_B", "0") != "1"
    if args.only in ("c2c", "r2c", "r2c64"):
        io = "r2c" if args.only == "r2c64" else args.only
        plan = ConvPlan("helmholtz", n=args.n, period=3, precision=prec, io=io,
                        batch_max=args.batch, kappa=20.0, compact=compact)
        dt = plan.cplx_dtype if args.only == "c2c" else plan.real_dtype
        u = torch.tensor(inputs.bump_sums(args.n, args.batch), dtype=dt, device="cuda")
    else:
        plan = ConvPlan("log", n=args.n, period=3, precision=prec, io="r2r", batch_max=args.batch,
                        compact=compact)
        u = torch.tensor(inputs.bump_sums(args.n, args.batch), dtype=plan.real_dtype, device="cuda")
    out = torch.empty(u.shape, dtype=plan.out_dtype(), device="cuda")
    for _ in range(args.warmup + args.steps):
        plan.apply(u, out=out)
    torch.cuda.synchronize()
    info = plan.info
    print(json.dumps({"case": args.only, "n": args.n, "batch": args.batch, "M": plan.M,
                      "threads_per_transform": info.threads_rows, "groups": info.groups_rows,
                      "radices": list(info.radices)[:info.nstages]}))


def serving_leg(count, seed=5):
    """Request mix (Poisson arrivals, mean 200/s): half convolutions, half Lippmann-Schwinger
    solves; n from {128, 256, 512, 1024, 2048} with weights .3/.3/.2/.15/.05; kernels from the
    five-kernel sweep; kappa ~ U[5, 60]; FP32 convolutions, mixed-precision LS (FP64 refinement to
    1e-10).  Submitted by a producer thread at the drawn arrival times; 150 GB budget."""
    import threading
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import Server
    reqs = inputs.serving_requests(count, rate=200.0, seed=seed)
    bufs = []
    for r in reqs:
        n = r["n"]
        if r["kind"] == "ls":
            m = torch.tensor(inputs.lippmann_contrast(n, "bump"), device="cuda")
            f = torch.tensor(inputs.plane_wave(n, r["kappa"]), device="cuda")
            bufs.append((m, f, torch.zeros_like(f)))
        else:
            u = torch.tensor(inputs.bump_sums(n, 1, seed=r["seed"])[0], dtype=torch.float32, device="cuda")
            cplx = r["kernel"] == "helmholtz"
            out = torch.empty((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda")
            bufs.append((u, out))
    # 4 LS worker streams: more run more solves at once but slow the plan builds and batches
    # queued beside them (p99 69 ms with 4, 96-116 ms with 8 on one box)
    srv = Server(mem_budget_bytes=150 << 30, max_inflight=64, conv_batch_max=16, ls_workers=4, compact=True)
    # warm-up, untimed, as a server does before it takes traffic: one request per convolution plan
    # of the mix (its five kernels at its five sizes) and one small LS solve, which load the
    # kernels' modules and make the convolution plans resident (every LS request of the mix has a
    # fresh kappa, so its plan is built on the request's path anyway)
    warm = []
    for n in inputs.SERVING_SIZES:
        u = torch.tensor(inputs.bump_sums(n, 1, seed=7)[0], dtype=torch.float32, device="cuda")
        for kern, kw in inputs.SWEEP_KERNELS:
            cplx = kern == "helmholtz"
            o = torch.empty((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda")
            warm.append((u, o, srv.submit_conv(u, o, kernel=kern, precision="fp32", io="r2c" if cplx else "r2r",
                                               **dict(kw))))
    m0 = torch.tensor(inputs.lippmann_contrast(128, "bump"), device="cuda")
    f0 = torch.tensor(inputs.plane_wave(128, 7.0), device="cuda")
    x0 = torch.zeros_like(f0)
    warm.append((m0, f0, srv.submit_ls(m0, f0, x0, 7.0, precision="fp32")))
    for w in warm:
        srv.wait(w[-1], timeout_s=600)
    st_warm = srv.stats()
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def producer():
        for i, r in enumerate(reqs):
            delay = r["t_arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            if r["kind"] == "ls":
                m, f, x = bufs[i]
                tickets[i] = srv.submit_ls(m, f, x, r["kappa"], precision="fp32")
            else:
                u, out = bufs[i]
                kw = dict(r["params"])
                io = "r2c" if r["kernel"] == "helmholtz" else "r2r"
                tickets[i] = srv.submit_conv(u, out, kernel=r["kernel"], precision="fp32", io=io, **kw)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    res = [srv.wait(t, timeout_s=600) for t in tickets]
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    ok = [r for r in res if r["status"] == "CONV_OK"]
    lat = sorted(r["latency_s"] for r in ok)
    lat_ls = sorted(r["latency_s"] for r, q in zip(res, reqs) if q["kind"] == "ls" and r["status"] == "CONV_OK")
    pct = lambda a, p: 1e3 * a[min(len(a) - 1, max(0, int(math.ceil(p * len(a))) - 1))] if a else None
    conv_res = [r for r, q in zip(res, reqs) if q["kind"] == "conv" and r["status"] == "CONV_OK"]
    return {"requests": count, "completed_ok": len(ok), "wall_s": wall,
            "conv_mean_batch": sum(r["batched_with"] for r in conv_res) / max(1, len(conv_res)),
            "requests_per_s": len(ok) / wall,
            "ls_solves_per_s": len(lat_ls) / wall, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
            "ls_p50_ms": pct(lat_ls, 0.5), "ls_p99_ms": pct(lat_ls, 0.99),
            "ls_max_rel_residual": max((r["rel_residual"] for r, q in zip(res, reqs) if q["kind"] == "ls"), default=None),
            "batches": stats["batches"] - st_warm["batches"],
            "batched_requests": stats["batched_requests"] - st_warm["batched_requests"],
            "plans_built": stats["plans_built"] - st_warm["plans_built"], "plans_evicted": stats["plans_evicted"],
            "ls_workers": 4, "mix": "50% conv / 50% LS, Poisson 200/s",
            "warm_up": "untimed: one request per convolution plan of the mix (25) and one LS solve at n = 128"}


def served_ls_burst(count, seed=5):
    """The LS requests of the serving mix (n from the mix's sizes, kappa ~ U[5, 60], tolerance
    1e-10), all submitted at once to a server whose plans are already resident (one untimed pass
    first): saturated solves/s of the served mixed-precision path against the served all-FP64
    path, with the final relative residual of each."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import Server
    reqs = [r for r in inputs.serving_requests(count, rate=200.0, seed=seed) if r["kind"] == "ls"]
    bufs = []
    for r in reqs:
        m = torch.tensor(inputs.lippmann_contrast(r["n"], "bump"), device="cuda")
        f = torch.tensor(inputs.plane_wave(r["n"], r["kappa"]), device="cuda")
        bufs.append((m, f, torch.zeros_like(f)))
    out = {"solves": len(reqs), "sizes": sorted(set(r["n"] for r in reqs))}
    for prec, name in (("fp32", "mixed"), ("fp64", "fp64")):
        srv = Server(mem_budget_bytes=150 << 30, max_inflight=64, conv_batch_max=16, ls_workers=8, compact=True)
        for timed in (False, True):
            for b in bufs:
                b[2].zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tickets = [srv.submit_ls(m, f, x, r["kappa"], precision=prec) for r, (m, f, x) in zip(reqs, bufs)]
            res = [srv.wait(t, timeout_s=600) for t in tickets]
            wall = time.perf_counter() - t0
        srv.close()
        lat = sorted(r["latency_s"] for r in res if r["status"] == "CONV_OK")
        pct = lambda a, p: 1e3 * a[min(len(a) - 1, max(0, int(math.ceil(p * len(a))) - 1))] if a else None
        out[name] = {"solves_per_s": len(lat) / wall, "wall_s": wall, "completed_ok": len(lat),
                     "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                     "max_rel_residual": max(r["rel_residual"] for r in res)}
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def served_conv_burst(count, seed=6):
    """The convolution requests of the serving mix (n from the mix's sizes, kernels of the sweep,
    Helmholtz kappa ~ U[5, 60]; FP32), all submitted at once to a server whose plans are already
    resident (one untimed pass first): saturated throughput with continuous batching by transform
    shape (batch up to 16) against the same server with batches of one."""
    import torch
    from paper_2107_03958_gb300 import inputs
    from paper_2107_03958_gb300.api import Server
    reqs = [r for r in inputs.serving_requests(count, rate=200.0, seed=seed, ls_fraction=0.0)]
    bufs = []
    for r in reqs:
        n = r["n"]
        u = torch.tensor(inputs.bump_sums(n, 1, seed=r["seed"])[0], dtype=torch.float32, device="cuda")
        cplx = r["kernel"] == "helmholtz"
        bufs.append((u, torch.empty((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda")))
    out = {"requests": len(reqs), "sizes": sorted(set(r["n"] for r in reqs))}
    for bmax, name in ((16, "batched"), (1, "unbatched")):
        srv = Server(mem_budget_bytes=150 << 30, max_inflight=64, conv_batch_max=bmax, ls_workers=1, compact=True)
        for timed in (False, True):
            torch.cuda.synchronize()
            st0 = srv.stats()
            t0 = time.perf_counter()
            tickets = []
            for r, (u, o) in zip(reqs, bufs):
                io = "r2c" if r["kernel"] == "helmholtz" else "r2r"
                tickets.append(srv.submit_conv(u, o, kernel=r["kernel"], precision="fp32", io=io, **dict(r["params"])))
            res = [srv.wait(t, timeout_s=600) for t in tickets]
            wall = time.perf_counter() - t0
            st1 = srv.stats()
        srv.close()
        lat = sorted(r["latency_s"] for r in res if r["status"] == "CONV_OK")
        pct = lambda a, p: 1e3 * a[min(len(a) - 1, max(0, int(math.ceil(p * len(a))) - 1))] if a else None
        out[name] = {"conv_per_s": len(lat) / wall, "wall_s": wall, "completed_ok": len(lat),
                     "batches": st1["batches"] - st0["batches"],
                     "batched_requests": st1["batched_requests"] - st0["batched_requests"],
                     "mean_batch": sum(r["batched_with"] for r in res) / max(1, len(res)),
                     "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99)}
    out["batched_over_unbatched"] = out["batched"]["conv_per_s"] / out["unbatched"]["conv_per_s"]
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.only:
        import paper_2107_03958_gb300.build as B
        B.build()
        profile_case(args)
        return
    import torch
    import paper_2107_03958_gb300.build as B
    B.build()
    from paper_2107_03958_gb300.api import measure_peaks
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, threads, secs = cpu_oracle_rate(args.n)
        cpu = {"value": rate, "unit": "conv/s", "cores": threads, "kind": "oracle",
               "sample": "1 of the step's 80 convolutions (density 0, log kernel, n=%d, b=3), FP64 C "
                         "oracle, %.1f s" % (args.n, secs)}

    peaks = measure_peaks(1 << 30)
    hbm, hbm_src = hbm_peak()
    alu_peak = {"fp64": peaks["fp64_tflops"], "fp32": peaks["fp32_tflops"]}
    alu_nominal = {"fp64": FP64_NOMINAL_TFLOPS, "fp32": FP32_NOMINAL_TFLOPS}

    # headline: the sweep at args.precision, device-resident inputs, per-pass events
    prec = args.precision
    clocks = ClockSampler(local)
    barrier(ws)
    clocks.start()
    head = sweep_leg(args.n, args.batch, prec, args.steps, args.warmup, stream, timing=True)
    clk = clocks.stop()
    ms = max_over_ranks(ws, head["ms"])
    convs = 5 * args.batch * args.steps
    value = job_throughput(ws, convs, ms)
    roofline = sweep_roofline(head, args.batch, prec, alu_peak[prec], alu_nominal[prec], hbm, hbm_src)
    roofline["live_peaks"] = peaks
    roofline["hbm_period3_schedule"] = period3_view(args.n, args.batch, prec, roofline["avg_launch_ms"],
                                                    ms / args.steps, hbm)
    head.pop("plans")
    torch.cuda.empty_cache()

    # end to end: pinned host inputs and results through conv_apply_host_multi, copies timed
    e2e_steps = max(3, args.steps // 2)
    e2e_run = e2e_leg(args.n, args.batch, e2e_steps, max(3, args.warmup), precision=prec)
    e2e_ms = max_over_ranks(ws, e2e_run["ms"])
    e2e = {"value": ws * 5 * args.batch * e2e_steps / (e2e_ms * 1e-3), "unit": "conv/s",
           "h2d_bytes_per_step": e2e_run["h2d"], "d2h_bytes_per_step": e2e_run["d2h"],
           "api": "conv_apply_host_multi (pinned host buffers; one upload per chunk for the five plans)"}

    # the other precision's sweep, same workload
    other = "fp32" if prec == "fp64" else "fp64"
    k_o = args.steps if other == "fp32" else max(2, args.steps // 4)
    orun = sweep_leg(args.n, args.batch, other, k_o, min(args.warmup, 3), stream, timing=True)
    o_ms = max_over_ranks(ws, orun["ms"])
    o_roof = sweep_roofline(orun, args.batch, other, alu_peak[other], alu_nominal[other], hbm, hbm_src)
    o_roof["hbm_period3_schedule"] = period3_view(args.n, args.batch, other, o_roof["avg_launch_ms"], o_ms / k_o, hbm)
    orun.pop("plans")
    torch.cuda.empty_cache()
    o_e2e = e2e_leg(args.n, args.batch, max(3, k_o // 2), 3, precision=other)
    sibling = {"value": job_throughput(ws, 5 * args.batch * k_o, o_ms), "unit": "conv/s", "dtype": other[:1] + other[2:],
               "steps": k_o, "ms_per_step": o_ms / k_o,
               "tolerance_vs_oracle": 2e-6 if other == "fp32" else 1e-12,
               "roofline": o_roof,
               "e2e": {"value": ws * 5 * args.batch * max(3, k_o // 2) / (max_over_ranks(ws, o_e2e["ms"]) * 1e-3),
                       "unit": "conv/s", "h2d_bytes_per_step": o_e2e["h2d"], "d2h_bytes_per_step": o_e2e["d2h"]}}

    # error of density 0 of each kernel of both sweeps against the FP64 oracle (outside every
    # timed region)
    err = None
    if rank == 0 and not args.no_oracle_check:
        t0 = time.perf_counter()
        refs = oracle_reference(head["u0"], args.n)
        err = {"max_rel_linf": errors_vs_oracle(head["out0"], refs),
               "tolerance": 1e-12 if prec == "fp64" else 2e-6,
               "sample": "density 0 of the last timed step, each kernel, against the FP64 C oracle's "
                         "full period-3 FFT convolution (%.0f s)" % (time.perf_counter() - t0)}
        sibling["err_vs_oracle"] = {"max_rel_linf": errors_vs_oracle(orun["out0"], refs)}
        del refs
    del head["out0"], orun["out0"]

    extras = {other: sibling}
    if not args.no_extras:
        kb = max(3, args.steps // 2)
        pb = sweep_leg(args.n, args.batch, "fp32", kb, args.warmup, stream, timing=True, compact=False)
        pb_ms = max_over_ranks(ws, pb["ms"])
        rpb = [(p, t) for p, t in zip(pb["plans"], pb["passes"]) if p.io == "r2r"]
        cpb = sum(t[0][1] for _, t in rpb) / sum(t[1] for _, t in rpb)
        bpb = r2r_bytes(rpb[0][0], args.batch)
        extras["fp32_period_b"] = {
            "value": job_throughput(ws, 5 * args.batch * kb, pb_ms), "unit": "conv/s", "steps": kb,
            "ms_per_step": pb_ms / kb, "transform_len": rpb[0][0].info.transform_len,
            "roofline_cols": {"bound": "hbm", "achieved": bpb / (cpb * 1e-3) / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": bpb / (cpb * 1e-3) / 1e9 / hbm,
                              "algorithmic_bytes_per_launch": bpb, "avg_launch_ms": cpb}}
        # the non-integer period b = 5/2 (M = 2.5 n = 10240: radix-5 runtime stages), FP32
        p25 = sweep_leg(args.n, args.batch, "fp32", kb, args.warmup, stream, timing=True, compact=False,
                        period=2.5)
        p25_ms = max_over_ranks(ws, p25["ms"])
        r25 = [(p, t) for p, t in zip(p25["plans"], p25["passes"]) if p.io == "r2r"]
        c25 = sum(t[0][1] for _, t in r25) / sum(t[1] for _, t in r25)
        b25 = r2r_bytes(r25[0][0], args.batch)
        extras["fp32_period_2.5"] = {
            "value": job_throughput(ws, 5 * args.batch * kb, p25_ms), "unit": "conv/s", "steps": kb,
            "ms_per_step": p25_ms / kb, "transform_len": r25[0][0].info.transform_len,
            "roofline_cols": {"bound": "hbm", "achieved": b25 / (c25 * 1e-3) / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": b25 / (c25 * 1e-3) / 1e9 / hbm,
                              "algorithmic_bytes_per_launch": b25, "avg_launch_ms": c25}}
        del p25, r25
        torch.cuda.empty_cache()
        n2 = args.n // 2
        l2 = sweep_leg(n2, args.batch, "fp32", args.steps, args.warmup, stream)
        l2_ms = max_over_ranks(ws, l2["ms"])
        l2t = sweep_leg(n2, args.batch, "fp32", 3, 1, stream, timing=True)
        extras["fp32_n%d" % n2] = {"value": ws * 5 * args.batch * args.steps / (l2_ms * 1e-3),
                                   "unit": "conv/s", "ms_per_step": l2_ms / args.steps,
                                   "roofline_cols": cols_roofline(l2t, args.batch, alu_peak["fp32"], hbm,
                                                                  "measured FP32 FMA microbenchmark")}
        k64b = max(2, args.steps // 3)
        f64b = sweep_leg(n2, args.batch, "fp64", k64b, 1, stream, timing=True)
        f64b_ms = max_over_ranks(ws, f64b["ms"])
        extras["fp64_n%d" % n2] = {"value": ws * 5 * args.batch * k64b / (f64b_ms * 1e-3), "unit": "conv/s",
                                   "ms_per_step": f64b_ms / k64b, "steps": k64b,
                                   "roofline_cols": cols_roofline(f64b, args.batch, peaks["fp64_tflops"], hbm,
                                                                  "measured FP64 FMA microbenchmark")}
        extras["fp32_n8192"] = n8192_leg(5, stream, hbm, alu_peak["fp32"])
        extras["ls"] = ls_leg(512, 40.0, 5, stream)
        extras["ls_larger"] = [ls_leg(1024, 40.0, 3, stream), ls_leg(2048, 40.0, 3, stream)]
        extras["ls_multi_rhs"] = ls_multi_leg(512, 40.0, 8, 3, stream)
        extras["mixed_group"] = group_leg(50, stream)
        from paper_2107_03958_gb300.api import measure_tc_stage
        tcs = measure_tc_stage(4000)
        tcs["what"] = ("one radix-16 stage (Ns = 16) of an FP32 length-8192 column, one column per SM in shared "
                       "memory: CUDA-core butterflies vs a tcgen05 DFT-matrix product (BF16 hi+lo, 3 products, "
                       "FP32 accumulation); microseconds per stage per column")
        tcs["tensor_over_cuda_core"] = tcs["us_tensor"] / tcs["us_cuda_core"]
        extras["tc_stage"] = tcs
        extras["serving"] = serving_leg(2000)
        extras["shared_rows"] = {
            "fp64": shared_rows_leg(args.n, args.batch, "fp64", max(2, args.steps // 4), 2, stream),
            "fp32": shared_rows_leg(args.n, args.batch, "fp32", args.steps, 3, stream),
            "note": "the same 80-convolution sweep with pass 1 computed once for the five kernels"}
        torch.cuda.empty_cache()
        extras["served_ls_burst"] = served_ls_burst(80)
        extras["served_conv_burst"] = served_conv_burst(400)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "conv/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
                "data": "synthetic", "config": workload_config(args), "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": head["launches"],
                "err_vs_oracle": err}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
