"""Benchmark of the tiled sparse LBM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A benchmark step is one LBM time step (stage neighbourhood, gather, collide,
store, swap) over the whole synthetic geometry; every 100 steps the FP64
mass / momentum / residual reduction runs as well.  The default workload is
the D3Q19 FP64 sphere pack: 256^3 lattice, 4^3 tiles, 30% fluid, tau 0.6,
force 1e-6 along periodic x.  The metric is MLUPS over fluid nodes (Eq. 43 of
the paper counts only non-solid nodes) and the fraction of the HBM roofline
(B_node = 304 B per update, Eq. 10).

With N > 1 (torchrun) the geometry is split into slabs of tile layers along
z, one per GPU, whose ghost layers are exchanged with NCCL after every step
(``--parallel split``, strong scaling), or every rank runs an independent
replica (``--parallel replicas``, weak scaling).  ``--impl reference`` times
the FP64 CPU oracle instead, on the host cores, on a 64^3 crop of the same
workload.  At N = 1 the line also carries the second half of the metric,
``steady``: time to residual 1e-6 of every storage form and of the warm
start against the plain FP64 solve from rest, on held-out 64^3 packs.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1703_08015_gb300 import geometry as geo  # noqa: E402
from paper_1703_08015_gb300 import perfmodel as pm  # noqa: E402

STATS_EVERY = 100
B_NODE = {9: pm.B_node(9, 8), 19: pm.B_node(19, 8)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="d3q19_spheres_256")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arith", default="auto", choices=["auto", "f64", "fixed", "ff", "ff_table"],
                    help="FP64 arithmetic: auto = ff, the staged tile-map step; ff_table = the per-node "
                         "gather table (the connectivity-matrix scheme of Sec. 2.3.1)")
    ap.add_argument("--storage", default="f64", choices=["f64", "f32", "f32s", "f16s"])
    ap.add_argument("--layout", default="t2c", choices=["t2c", "tgb"],
                    help="two PDF copies (T2C) or one copy with ghost buffers (TGB)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-steady", action="store_true", help="skip the time-to-steady-state part of the line")
    ap.add_argument("--steady-seconds", type=float, default=40.0,
                    help="time budget of the time-to-steady-state part (held-out packs are added until it is spent)")
    ap.add_argument("--mode", default="throughput", choices=["throughput", "steady", "batch", "conv"])
    ap.add_argument("--parallel", default="split", choices=["split", "replicas"],
                    help="N > 1 GPUs: split the geometry into slabs of tile layers with ghost layers exchanged "
                         "over NCCL every step (strong scaling), or run independent replicas (weak scaling)")
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--max-steps", type=int, default=100000)
    ap.add_argument("--target", type=float, default=1e-6)
    ap.add_argument("--weights", default=None, help="warm-start network weights (steady mode)")
    return ap.parse_args()


ISSUE_PEAK = 152 * 4 * 2.07e9  # warp instructions per second: SMs x schedulers x 1/clock x max SM clock


def issue_roofline(args, arith_name, n_fluid, step_ms):
    """Instruction-issue view of the step kernel (the FP64 and FP32 steps are
    bound by issue and latency, not by HBM): warp instructions per launch from
    the committed ncu count per fluid node, over the measured kernel time,
    against one instruction per scheduler per clock."""
    if args.layout != "t2c":
        return None
    e = committed_profile(args.workload, arith_name if args.storage == "f64" else args.storage)
    per_node = e.get("warp_instructions_per_node")
    if not per_node:
        return None
    achieved = per_node * n_fluid / (step_ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": ISSUE_PEAK, "unit": "warp instructions/s",
            "frac": achieved / ISSUE_PEAK, "warp_instructions_per_node": per_node,
            "peak_source": "152 SMs x 4 schedulers x 1 instruction/clock x 2.07 GHz"}


def replica_throughput(ms, n_fluid, steps, world, device):
    """Whole-job throughput of `world` independent replicas (one per GPU, each
    updating n_fluid nodes `steps` times): the slowest rank's time over all
    ranks' updates.  Returns (max time in ms, MLUPS)."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, n_fluid * steps * world / (ms_max * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


CLOCK_Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def _clock_rows(text):
    """(sm MHz, max MHz, active reasons) per nvidia-smi CSV row of CLOCK_Q."""
    out = []
    for r in csv.reader(io.StringIO(text)):
        if len(r) < 10:
            continue
        try:
            sm, smax = float(r[2]), float(r[3])
        except ValueError:
            continue
        out.append((sm, smax, {n for k, n in enumerate(CLOCK_REASONS) if r[6 + k].strip().lower() == "active"}))
    return out


def clock_snapshot(gpu_index):
    """One read-only nvidia-smi query of the SM clock and throttle reasons."""
    try:
        r = subprocess.run(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                            "-i", str(gpu_index)], capture_output=True, text=True, timeout=20)
        return _clock_rows(r.stdout)
    except (OSError, subprocess.SubprocessError):
        return []


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons around and during a
    window: one query just before it starts, a 20 ms sampling loop while it
    runs, one query just after it ends (all read-only)."""

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.before = clock_snapshot(gpu_index)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # the sampler is up before the window opens
        except OSError:
            self.proc = None

    def stop(self):
        during = []
        if self.proc is not None:
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            during = _clock_rows(out)
        after = clock_snapshot(self.gpu)
        rows = self.before + during + after
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        reasons = set().union(*(r[2] for r in rows))
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[-1][1],
                "reasons": sorted(reasons), "samples": len(rows), "samples_during": len(during),
                "sm_mhz_before": self.before[0][0] if self.before else None,
                "sm_mhz_after": after[0][0] if after else None,
                "how": "nvidia-smi query just before and just after the timed region, -lms 20 loop during it"}


STEP_SOURCES = {  # the sources each step kernel is built from
    "common": ("internal.h", "lattice.cuh", "tile.cuh", "tiling.cpp"),
    "ff_staged": ("collide_f64.cuh", "collide_ff.cuh", "step_ff.cu"),
    "ff_table_cm": ("collide_f64.cuh", "collide_ff.cuh", "step_ff_table.cu"),
    "fixed": ("collide_f64.cuh", "step_fixed.cu"),
    "f64": ("collide_f64.cuh", "step_f64.cu"),
    "f32": ("collide_f32.cuh", "step_f32.cu"),
}


def kernel_source_sha(kind="ff"):
    """Hash of the sources a step kernel is built from (a committed traffic
    figure is used only while they are unchanged)."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1703_08015_gb300", "csrc")
    for f in STEP_SOURCES["common"] + STEP_SOURCES[kind]:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def committed_profile(workload, arith):
    """The committed ncu figures of the step kernel for this workload, if they
    were taken on the current kernel sources (else {})."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        e = json.load(f).get(f"{workload}:{arith}")
    kind = arith if arith in STEP_SOURCES else "f32"
    if not e or e.get("kernel_source_sha") != kernel_source_sha(kind):
        return {}
    return e


def committed_traffic(workload, arith):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{arith}")
    kind = arith if arith in STEP_SOURCES else "f32"
    if not e or e.get("kernel_source_sha") != kernel_source_sha(kind):
        return None, None
    return e.get("dram_bytes_per_launch"), e.get("note")


def step_kernel_name(lat, a, storage, layout, arith_name):
    """The step kernel a bench line times, with the form of its gather."""
    lt = "D3Q19" if lat == 19 else "D2Q9"
    if layout == "tgb":
        return f"k_step_tgb<{lt},{a}> (single copy with ghost buffers, Fig. 4 layout, pull form)"
    if storage != "f64":
        store = {"f32": "StoreF32", "f32s": "StoreF32S", "f16s": "StoreF16S"}[storage]
        return (f"k_step_f32<{lt},{a},{store}> (tile-map T2C step of Fig. 5: neighbourhood staged per "
                "block; FP32 collision)")
    nt = a ** (3 if lat == 19 else 2)  # nodes per tile
    staged = (("per-tile neighbour records" if nt <= 64 else "neighbour indices and records") +
              f" staged per block of {128 if nt <= 256 else nt} nodes")
    return {"ff_staged": f"k_step_ff<{lt},{a}> (tile-map T2C step of Fig. 5: {staged}; float-float FP64 update)",
            "ff_table_cm": f"k_step_ff_table<{lt}> (per-node gather table built once: the connectivity-matrix "
                           "scheme of Sec. 2.3.1 on compact tiles, not the tile-map method; float-float FP64)",
            "fixed": f"k_step_fixed<{lt},{a}> (tile-map T2C step; 64-bit fixed-point FP64 update)",
            "f64": f"k_step_f64<{lt},{a}> (tile-map T2C step; native FP64 update)"}[arith_name]


def cpu_baseline(mask, params, seconds=10.0, min_steps=2):
    """The FP64 oracle, as it stands, on a 64^3 crop of the workload."""
    import oracle

    crop = np.ascontiguousarray(mask[:64, :64, :64]) if mask.shape[0] > 1 else np.ascontiguousarray(mask)
    lat = params["lattice"]
    per = params["periodic"]
    nf = int(crop.sum())

    def timed(nthreads, secs):
        f = oracle.init(lat, crop)
        g = np.empty_like(f)
        oracle.step(lat, crop, per, params["tau"], params["force"], f, out=g, nthreads=nthreads)  # warm-up
        n = 0
        t0 = time.perf_counter()
        while n < min_steps or time.perf_counter() - t0 < secs:
            oracle.step(lat, crop, per, params["tau"], params["force"], f, out=g, nthreads=nthreads)
            f, g = g, f
            n += 1
        return n, time.perf_counter() - t0

    n, dt = timed(0, seconds)
    n1, dt1 = timed(1, seconds / 3)
    return {"value": nf * n / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(0), "kind": "oracle",
            "value_1_thread": nf * n1 / dt1 / 1e6,
            "sample": f"{n} oracle steps on the {crop.shape[2]}x{crop.shape[1]}x{crop.shape[0]} corner "
                      f"crop ({nf} fluid nodes) of the workload, {dt:.1f} s on all threads; "
                      f"{n1} steps, {dt1:.1f} s on one thread (value_1_thread)"}


# Time-to-steady forms: (label, storage, start, period-2 filter[, storage that
# finishes the run once the residual of the first stops falling]); the first
# is the baseline every speedup is quoted against, the first filtered zero
# start the reference every error is measured against.
STEADY_CASES = [("f64_zero_plain", "f64", "zero", False), ("f64_zero", "f64", "zero", True),
                ("f64_warm", "f64", "warm", True), ("f32s_zero", "f32s", "zero", True),
                ("f32s_warm", "f32s", "warm", True), ("f16s_zero", "f16s", "zero", True, "f32s")]


def steady_summary(dev, budget_s=40.0, min_packs=4, max_packs=64, target=1e-6):
    """The second half of the metric: wall time to residual < target (checked
    every 100 steps with the FP64 reduction; tiling, initialisation and network
    inference inside the timing) on held-out 64^3 sphere packs (seed 2, never
    trained on), per form, against the plain FP64 solve from rest; packs are
    added until `budget_s` is spent."""
    from paper_1703_08015_gb300 import nn
    from paper_1703_08015_gb300 import warmstart

    net = nn.UNet.load(nn.WEIGHTS, device=dev) if os.path.exists(nn.WEIGHTS) else None
    cases = STEADY_CASES if net is not None else [c for c in STEADY_CASES if c[2] == "zero"]
    held, _ = nn.sample_geometries(max_packs, 2, 64)
    rows = []
    t0 = time.perf_counter()
    for m in held:
        rows += warmstart.evaluate(net, [m], cases, target=target, max_steps=60000, device=dev)
        if len(rows) >= min_packs and time.perf_counter() - t0 > budget_s:
            break
    summ = warmstart.summarize(rows, cases)
    forms = {}
    for label, form, start, filt, *fin in cases:
        e = summ.get(label)
        if not e:
            continue
        forms[label] = {"storage": form, "start": start, "period2_filter": filt,
                        "finish_storage": fin[0] if fin else None,
                        "converged": e["converged"], "steps_median": e["steps_median"],
                        "seconds_total": e["seconds_total"],
                        "speedup_vs_fp64_zero_start": e["speedup_vs_" + cases[0][0]],
                        "permeability_rel_err_max": e["permeability_rel_err_max"],
                        "u_rel_err_median": e["u_rel_err_median"], "switched_to_finish": e.get("switched", 0)}
    ok = [k for k, v in forms.items() if k != cases[0][0] and v["permeability_rel_err_max"] <= 1e-3]
    best = max(ok, key=lambda k: forms[k]["speedup_vs_fp64_zero_start"]) if ok else None
    return {"metric": f"time to residual < {target:g} vs the plain FP64 zero start", "target_residual": target,
            "workload": f"{len(rows)} held-out 64^3 sphere packs (radius 4-12, fluid 10-60 %, seed 2), "
                        "tau 0.6, F 1e-6 along periodic x, residual every 100 steps",
            "packs": len(rows), "all_converged": summ.get("all_converged", 0),
            "permeability_reference": "filtered FP64 zero start (f64_zero)",
            "permeability_rel_err_bound": 1e-3, "best_form": best,
            "best_speedup_vs_fp64_zero_start": forms[best]["speedup_vs_fp64_zero_start"] if best else None,
            "forms": forms, "seconds": time.perf_counter() - t0,
            "warm_start_weights": os.path.basename(nn.WEIGHTS) if net is not None else None}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    mask, params, info = geo.workload(args.workload)
    crop = np.ascontiguousarray(mask[:64, :64, :64]) if mask.shape[0] > 1 else np.ascontiguousarray(mask)
    lat = params["lattice"]
    per = params["periodic"]
    f = oracle.init(lat, crop)
    g = np.empty_like(f)
    for _ in range(args.warmup):
        oracle.step(lat, crop, per, params["tau"], params["force"], f, out=g)
        f, g = g, f
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(lat, crop, per, params["tau"], params["force"], f, out=g)
        f, g = g, f
    dt = time.perf_counter() - t0
    nf = int(crop.sum())
    v = nf * args.steps / dt / 1e6
    # the same metric, unit and workload as our arm; each step a bounded sample of it
    line = {"impl": "reference",
            "metric": "D3Q19 sparse MLUPS + % HBM roofline" if lat == 19 else "D2Q9 sparse MLUPS + % HBM roofline",
            "value": v, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": f"D{3 if lat == 19 else 2}Q{lat}",
                       "size": list(mask.shape[::-1]), "tile": params["tile_a"], "storage": "f64",
                       "sample_crop": list(crop.shape[::-1]), "sample_fluid_nodes": nf},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(0), "kind": "oracle",
                             "sample": f"each step: one oracle step on the 64^3 corner crop ({nf} fluid nodes)"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_split(args):
    """N GPUs on one geometry: slabs of tile layers along z, one ghost tile
    layer per neighbour, exchanged after every step with NCCL send/recv into
    the receiver's own PDF buffer (slab.py); value = all fluid updates over
    the slowest rank's time (strong scaling: the workload is fixed)."""
    import torch
    import torch.distributed as dist

    from paper_1703_08015_gb300 import lbm
    from paper_1703_08015_gb300 import slab

    rank, world, local = dist_env()
    dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mask, params, info = geo.workload(args.workload)
    lat, a = params["lattice"], params["tile_a"]
    arith = {"auto": lbm.LBM_ARITH_AUTO, "f64": lbm.LBM_ARITH_F64, "fixed": lbm.LBM_ARITH_FIXED,
             "ff": lbm.LBM_ARITH_FF, "ff_table": lbm.LBM_ARITH_FF_TABLE}[args.arith]
    s = slab.SlabSolver(mask, lat, a, params["periodic"], params["tau"], params["force"], rank, world,
                        slab.TorchDistComm(dist), arith=arith, device=dev)
    n_fluid = int(mask.sum())

    def reduce_stats(v):
        t = torch.tensor(v, dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        return t.tolist()

    s.step(max(3, args.warmup))
    s.stats(residual=True, all_reduce=reduce_stats)
    dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.solver.stream)
    left = args.steps
    while left > 0:
        k = min(STATS_EVERY, left)
        s.step(k)
        left -= k
        if k == STATS_EVERY:
            s.stats(residual=True, all_reduce=reduce_stats)
    e1.record(s.solver.stream)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms_max, value = replica_throughput(e0.elapsed_time(e1), n_fluid, args.steps, 1, dev)
    t = torch.tensor([ms_max], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = n_fluid * args.steps / (ms_max * 1e-3) / 1e6
    part = s.part
    s.close()
    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    achieved = n_fluid * pm.B_node(lat, 8) / (ms_max / args.steps * 1e-3) / 1e9
    print(json.dumps({
        "metric": "D3Q19 sparse MLUPS + % HBM roofline" if lat == 19 else "D2Q9 sparse MLUPS + % HBM roofline",
        "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"D{3 if lat == 19 else 2}Q{lat}",
                   "size": list(mask.shape[::-1]), "tile": a, "fluid_nodes": n_fluid,
                   "parallelism": f"split{world}: slabs of tile layers along z, one ghost layer per neighbour, "
                                  "NCCL send/recv every step",
                   "rank0_layers": [part["lo"], part["hi"]], "stats_every": STATS_EVERY,
                   "l2": "inputs larger than L2", "geometry": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"] * world, "unit": "GB/s",
                     "frac": achieved / (peaks["hbm_gbs"] * world), "traffic": None,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs) x {world} GPUs",
                     "kernel": step_kernel_name(lat, a, "f64", "t2c", "ff_staged"),
                     "note": "whole-job time including the ghost-layer exchange"},
        "clocks": clocks, "gpu_launches": args.steps}))


def run_ours(args):
    import torch

    from paper_1703_08015_gb300 import lbm

    rank, world, local = dist_env()
    if world > 1 and args.parallel == "split":
        return run_split(args)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mask, params, info = geo.workload(args.workload)
    lat, a = params["lattice"], params["tile_a"]
    arith = {"auto": lbm.LBM_ARITH_AUTO, "f64": lbm.LBM_ARITH_F64, "fixed": lbm.LBM_ARITH_FIXED,
             "ff": lbm.LBM_ARITH_FF, "ff_table": lbm.LBM_ARITH_FF_TABLE}[args.arith]
    storage = {"f64": lbm.LBM_STORE_F64, "f32": lbm.LBM_STORE_F32, "f32s": lbm.LBM_STORE_F32S,
               "f16s": lbm.LBM_STORE_F16S}[args.storage]
    layout = {"t2c": lbm.LBM_LAYOUT_T2C, "tgb": lbm.LBM_LAYOUT_TGB}[args.layout]
    solver = lbm.Solver(mask, lat, a, params["periodic"], params["tau"], params["force"], arith=arith,
                        storage=storage, layout=layout, device=dev)
    stream = solver.stream
    n_fluid = int(solver.tiling.n_fluid)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(3, args.warmup) // 20 + 1):
        solver.step(20)
    solver.stats(residual=True)
    barrier()

    sampler = ClockSampler(local)
    ev = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    launches = 0
    t_start.record(stream)
    left = args.steps
    while left > 0:
        k = min(STATS_EVERY, left)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(k)
        e1.record(stream)
        ev.append((e0, e1, k))
        launches += k
        left -= k
        if k == STATS_EVERY:
            st = lbm.lbm_stats()
            lbm.lbm_moments(solver.ctx, None, None, st, lbm.LBM_STATS_RESIDUAL, solver._s())
            launches += 2
    t_end.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end)
    step_ms = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / args.steps
    ms_max, value = replica_throughput(ms, n_fluid, args.steps, world, dev)
    # "ff_staged": the float-float tile-map step (the default, --arith auto or ff);
    # "ff_table_cm": the float-float step through the per-node gather table
    arith_name = {lbm.LBM_ARITH_AUTO: "ff_staged", lbm.LBM_ARITH_FIXED: "fixed", lbm.LBM_ARITH_F64: "f64",
                  lbm.LBM_ARITH_FF: "ff_staged", lbm.LBM_ARITH_FF_TABLE: "ff_table_cm"}[arith]
    tiling = solver.tiling
    solver.close()
    del solver
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(mask, params, args.steps, arith, dev, world, storage)

    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    s_d = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2}[args.storage]
    bytes_per_launch = n_fluid * pm.B_node(lat, s_d)
    achieved = bytes_per_launch / (step_ms * 1e-3) / 1e9
    traffic, tnote = (committed_traffic(args.workload, arith_name if args.storage == "f64" else args.storage)
                      if args.layout == "t2c" else (None, None))
    dev_bytes = int(tiling.pdf_bytes) + (int(tiling.ghost_bytes) if args.layout == "tgb" else int(tiling.pdf_bytes))
    tiling_stats = {"n_ftiles": int(tiling.n_ftiles), "n_tiles": int(tiling.n_tiles),
                    "phi": n_fluid / mask.size,
                    "phi_t": n_fluid / (tiling.n_ftiles * a ** (3 if lat == 19 else 2))}
    line = {
        "metric": "D3Q19 sparse MLUPS + % HBM roofline" if lat == 19 else "D2Q9 sparse MLUPS + % HBM roofline",
        "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "f32s": "f32", "f16s": "f16+f32"}[args.storage],
        "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"D{3 if lat == 19 else 2}Q{lat}",
                   "size": list(mask.shape[::-1]), "tile": a, "fluid_nodes": n_fluid, **tiling_stats,
                   "tau": params["tau"], "force": params["force"], "storage": args.storage,
                   "arith": arith_name if args.storage == "f64" else "f32",
                   "gather_table_bytes": ((lat + 1) * 4 * n_fluid
                                          if args.storage == "f64" and arith_name == "ff_table_cm" else 0),
                   "stats_every": STATS_EVERY, "parallelism": "replicas" if world > 1 else "single",
                   "layout": args.layout,
                   "pdf_device_bytes": dev_bytes,
                   "l2": (f"inputs larger than L2 (PDF state {dev_bytes / 1e9:.2f} GB, L2 129 MB)"
                          if dev_bytes > 129e6 else
                          f"L2-resident small case (PDF state {dev_bytes / 1e6:.1f} MB < L2 129 MB): "
                          "a latency figure, not an HBM measurement"),
                   "geometry": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": step_kernel_name(lat, a, args.storage, args.layout, arith_name),
                     "bytes_per_launch": bytes_per_launch,
                     "step_kernel_ms": step_ms, "traffic_note": tnote},
        "issue_roofline": issue_roofline(args, arith_name, n_fluid, step_ms),
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": e2e,
        "model_overheads": pm.predictions(lat, 8, a, 3 if lat == 19 else 2, tiling_stats["phi"],
                                          tiling_stats["phi_t"],
                                          tiling.n_tiles / max(1, tiling.n_ftiles)),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mask, params)
    if world == 1 and not args.no_steady and lat == 19 and args.storage == "f64" and args.layout == "t2c":
        line["steady"] = steady_summary(dev, args.steady_seconds)
    print(json.dumps(line))


def run_e2e(mask, params, steps, arith, dev, world, storage=0):
    """Same metric through the C ABI from host buffers: pinned host mask ->
    lbm_init (tiling + upload + equilibrium fill), the timed steps with the
    stats read back every 100 steps, and rho/u fields back to host memory."""
    import torch

    from paper_1703_08015_gb300 import lbm

    lat, a = params["lattice"], params["tile_a"]
    p = lbm.make_params(lat, mask.shape, a, params["periodic"], params["tau"], params["force"], arith=arith,
                        storage=storage)
    info, _, _ = lbm.lbm_build_tilemap(p, mask, want_map=False, want_nbr=False)
    nbytes = max(int(info.pdf_bytes), 256)
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    host_mask = torch.from_numpy(np.ascontiguousarray(mask)).pin_memory()
    d = 3 if lat == 19 else 2
    rho = torch.empty(mask.shape, dtype=torch.float64).pin_memory()
    u = torch.empty((d,) + mask.shape, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    s = ctypes_stream(stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx = lbm.lbm_init(p, host_mask.numpy(), bufs[0], bufs[1], nbytes, None, None, s)
    left = steps
    n_stats = 0
    while left > 0:
        k = min(STATS_EVERY, left)
        lbm.lbm_step(ctx, k, s)
        left -= k
        st = lbm.lbm_stats()
        lbm.lbm_moments(ctx, None, None, st, 0, s)
        n_stats += 1
    lbm.lbm_moments(ctx, rho.numpy(), u.numpy(), None, 0, s)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    lbm.lbm_free(ctx)
    words = (a ** (3 if lat == 19 else 2) + 63) // 64
    h2d = int(info.n_ftiles) * (int(info.nbr_per_tile) * 4 + words * 8 + 12)  # tile tables uploaded
    d2h = rho.numel() * 8 + u.numel() * 8 + n_stats * 64
    return {"value": int(info.n_fluid) * steps * world / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": dt, "includes": "host tiling, table upload, equilibrium fill, steps, stats, rho/u readback"}


def ctypes_stream(stream):
    import ctypes

    return ctypes.c_void_p(stream.cuda_stream)


def run_steady(args):
    """Time to steady state (residual below --target, checked every 100 steps
    with the FP64 reduction) on one GPU: the plain FP64 solve from rest (the
    baseline), then every storage form with the period-2 filter
    (lbm_filter_period2 after each residual check) and, when trained weights
    are present, started from the warm-start network's prediction.  Errors of
    every form against the filtered FP64 zero start."""
    import torch

    from paper_1703_08015_gb300 import lbm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mask, params, info = geo.workload(args.workload)
    lat, a = params["lattice"], params["tile_a"]
    nu = (params["tau"] - 0.5) / 3.0
    fx = params["force"][0]
    net = None
    weights = args.weights or os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1703_08015_gb300",
                                           "weights", "unet_spheres64.npz")
    if lat == 19 and os.path.exists(weights) and all(n % 8 == 0 for n in mask.shape):
        from paper_1703_08015_gb300 import nn

        net = nn.UNet.load(weights, device=dev)
    S = lbm
    forms = [("f64", S.LBM_STORE_F64, False, False), ("f64_p2", S.LBM_STORE_F64, True, False),
             ("f32s", S.LBM_STORE_F32S, False, False), ("f32s_p2", S.LBM_STORE_F32S, True, False),
             ("f32_p2", S.LBM_STORE_F32, True, False), ("f16s_p2", S.LBM_STORE_F16S, True, False)]
    if net is not None:
        forms += [("f64_warm_p2", S.LBM_STORE_F64, True, True), ("f32s_warm_p2", S.LBM_STORE_F32S, True, True)]
    res, fields = {}, {}
    fl = mask.astype(bool)
    for name, storage, filt, warm in forms:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rho0 = u0 = None
        if warm:
            rho0, u0 = nn.predict_fields(net, mask, fx, nu)
        s = lbm.Solver(mask, lat, a, params["periodic"], params["tau"], params["force"], storage=storage,
                       rho_init=rho0, u_init=u0, device=dev)
        st0, _ = s.stats(residual=True)
        n, st, hist, n_filter = 0, st0, [], 0
        while n < args.max_steps:
            s.step(STATS_EVERY)
            n += STATS_EVERY
            st, rc = s.stats(residual=True)
            hist.append(st.residual)
            if rc != 0 or st.residual < args.target:
                break
            if filt:
                s.filter_period2()
                n_filter += 1
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        rho, u, st_f, _ = s.moments()
        s.close()
        k = nu * float(np.sum(u[0][fl])) / mask.size / fx if fx else None  # superficial-velocity permeability
        fields[name] = u[:, fl]
        res[name] = {"steps": n, "filters": n_filter, "seconds": dt, "converged": bool(st.residual < args.target),
                     "final_residual": st.residual, "mlups": int(st.n_fluid) * n / dt / 1e6,
                     "permeability": k, "mass_drift": abs(st.mass - st0.mass) / st0.mass,
                     "residual_floor": float(min(hist)) if hist else None}
    ref = fields["f64_p2"]
    for name in res:
        d = fields[name] - ref
        res[name]["velocity_l2_rel_err_vs_f64_p2"] = float(np.sqrt(np.sum(d * d) / np.sum(ref * ref)))
        if res["f64_p2"]["permeability"]:
            res[name]["permeability_rel_err_vs_f64_p2"] = abs(res[name]["permeability"] /
                                                              res["f64_p2"]["permeability"] - 1)
        res[name]["speedup_vs_f64"] = res["f64"]["seconds"] / res[name]["seconds"]
    ok = [kk for kk, r in res.items() if kk != "f64" and r["converged"] and
          r.get("permeability_rel_err_vs_f64_p2", 1.0) <= 1e-3]
    best = min(ok, key=lambda kk: res[kk]["seconds"]) if ok else None
    if rank == 0:
        print(json.dumps({"metric": "time to steady state (residual < %g) vs plain FP64" % args.target,
                          "value": res["f64"]["seconds"] / res[best]["seconds"] if best else None,
                          "unit": "x speedup of the fastest form (permeability within 1e-3)",
                          "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "best_form": best,
                          "config": {"workload": args.workload, "check_every": STATS_EVERY,
                                     "max_steps": args.max_steps, "geometry": info,
                                     "warm_start_weights": os.path.basename(weights) if net is not None else None},
                          "forms": res}))


def run_batch(args):
    """Many porous samples (64 by default, sides 32-160, 10-60% fluid) in one
    concatenated tile list, FP32-deviation storage, the mapping chosen by the
    autotuner; MLUPS over all samples and the FP32 HBM roofline (152 B)."""
    import torch

    from paper_1703_08015_gb300 import autotune
    from paper_1703_08015_gb300 import lbm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    masks, infos = geo.batch_workload(args.samples)
    storage = {"f64": lbm.LBM_STORE_F64, "f32": lbm.LBM_STORE_F32, "f32s": lbm.LBM_STORE_F32S,
               "f16s": lbm.LBM_STORE_F16S}[args.storage if args.storage != "f64" else "f32s"]
    per, tau, force = (1, 0, 0), 0.6, (1e-6, 0.0, 0.0)
    t0 = time.perf_counter()
    best, trials = autotune.tune(masks, 19, storage, per, tau, force)
    t_tune = time.perf_counter() - t0
    b = lbm.BatchSolver(masks, 19, best["tile_a"], per, tau, force, storage=storage,
                        block_nodes=best["block_nodes"], persistent=best["persistent"],
                        prefetch_blocks=best.get("prefetch_blocks", 0), device=dev)
    n_fluid = int(b.tiling.n_fluid)
    b.step(max(3, args.warmup))
    b.stats(residual=True)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ms = 0.0
    e0.record(b.stream)
    left, launches = args.steps, 0
    while left > 0:
        k = min(STATS_EVERY, left)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(b.stream)
        b.step(k)
        a1.record(b.stream)
        a1.synchronize()
        step_ms += a0.elapsed_time(a1)
        left -= k
        launches += k
        if k == STATS_EVERY:
            b.stats(residual=True)
            launches += 2 * len(masks)
    e1.record(b.stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    b.close()
    peaks, kind = load_peaks()
    s_d = 2 if storage == lbm.LBM_STORE_F16S else 4
    achieved = n_fluid * pm.B_node(19, s_d) / (step_ms / args.steps * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "batched D3Q19 MLUPS (FP32 storage, one launch per step over all samples)",
            "value": n_fluid * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(masks)} sphere packs, sides 32-160, 10-60% fluid",
                       "fluid_nodes": n_fluid, "n_ftiles": int(b.tiling.n_ftiles),
                       "pdf_bytes_per_copy": int(b.tiling.pdf_bytes), "mapping": best,
                       "autotune_seconds": t_tune, "autotune_trials_mlups": trials},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "peak_source": kind,
                         "step_kernel_ms": step_ms / args.steps},
            "clocks": clocks, "gpu_launches": launches}))


# the warm-start U-Net's 3x3x3 convolutions at batch 8 (side, cin, cout)
CONV_LAYERS = [(64, 16, 16), (64, 48, 16), (32, 16, 32), (32, 32, 32), (32, 96, 32), (16, 32, 64), (16, 64, 64),
               (16, 192, 64), (8, 64, 128), (8, 128, 128)]


def run_conv(args):
    """Time the network's convolutions through lbm_nn_conv3d (kernel picked by
    shape) and, where the shape allows, lbm_nn_conv3d_tc (tcgen05), and their
    weight gradients (lbm_nn_conv3d_wgrad); one JSON line with TFLOP/s per
    layer."""
    import torch

    from paper_1703_08015_gb300 import nn

    batch, reps = 8, max(args.steps // 100, 5)
    rows = []
    for side, cin, cout in CONV_LAYERS:
        x = torch.randn(batch, side, side, side, cin, device="cuda").to(torch.bfloat16)
        w = (torch.randn(27, cin, cout, device="cuda") * 0.05).to(torch.bfloat16)
        y = torch.empty(batch, side, side, side, cout, device="cuda", dtype=torch.bfloat16)
        row = {"layer": f"{batch}x{side}^3 {cin}->{cout}"}
        for name, f in (("auto", nn.lbm_nn_conv3d), ("tcgen05", nn.lbm_nn_conv3d_tc)):
            for _ in range(3):
                f(x, batch, side, side, side, cin, w, None, cout, 1, 1, y, None)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f(x, batch, side, side, side, cin, w, None, cout, 1, 1, y, None)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[name + "_us"] = ms * 1e3
            row[name + "_tflops"] = 2.0 * batch * side ** 3 * 27 * cin * cout / ms / 1e9
        # the weight gradient of the same layer (dy shaped like y, FP32 accumulators)
        dw = torch.zeros(27 * cin * cout, device="cuda")
        for _ in range(3):
            nn.lbm_nn_conv3d_wgrad(x, y, batch, side, side, side, cin, cout, 1, dw, None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            nn.lbm_nn_conv3d_wgrad(x, y, batch, side, side, side, cin, cout, 1, dw, None)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        row["wgrad_us"] = ms * 1e3
        row["wgrad_tflops"] = 2.0 * batch * side ** 3 * 27 * cin * cout / ms / 1e9
        rows.append(row)
    print(json.dumps({"metric": "warm-start U-Net 3x3x3 convolution TFLOP/s (BF16, FP32 accumulation)",
                      "unit": "TFLOP/s", "dtype": "bf16", "data": "synthetic", "layers": rows,
                      "tc_timeouts": nn.lbm_nn_tc_timeouts()}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "steady":
        run_steady(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "conv":
        run_conv(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
