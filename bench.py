#!/usr/bin/env python
"""Throughput of the EULBFS explicit step on GB300 (one JSON line on stdout).

Workload: the batched static-droplet freezing problem -- 64 domains with
sides drawn from {128, 192, 256, 384, 512} (6.76 M cells), FP32 arithmetic
with compensated H and C, every stage of every domain in one launch over a
tile work list.  A step is one full SSP-RK3 time step of every domain.
Metric: GCUPS = cells x steps / s / 1e9, whole job over all ranks.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With --gpus N > 1 (launched by torchrun) every rank advances its own batch
of 64 domains (independent problems, weak scaling, no data-path collective).
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

STAGES = 3
# Algorithmic HBM bytes per cell and time step of the FP32C path:
#  - compulsory: the state read once and written once per step, 7 planes of
#    4 B each way plus F_s^{n-1} read and written (a fully fused step);
#  - stage-by-stage: what a kernel per Runge-Kutta stage must move (stage
#    input, W^n at stages 2 and 3, output; F_s and dF_s/dt).
BYTES_COMPULSORY = {1: 64, 0: 96}
BYTES_STAGE_BY_STAGE = {1: 244, 0: 352}
# Counters of the FP32C and FP64 stage kernels from ncu captures of the
# 64-domain batch (6.80 M cells, work items of 128 rows, a 16-step launch
# (FP64: 2 steps), planar and axisymmetric): per cell and stage, FP32 (FP64)
# operations with an FMA counted as 2 and warp instructions issued; per
# cell and step, DRAM bytes.  They belong to one version of the kernel's sources: the
# SHA-256 of stage.cu + device_common.cuh + eulbfs_internal.h.  When the
# sources change, the counters are reported as stale (null) until they are
# captured again.
KERNEL_SOURCES = ("stage.cu", "device_common.cuh", "eulbfs_internal.h")
COUNTERS = {
    "sources_sha256": "cbface8b97d14d2489ffbb3e171fe71d595a2fff85d003d3b12838e4224168c8",
    "fp32_flops_per_cell_stage": {"rz": 942.3, "xy": 905.0},
    "warp_inst_per_cell_stage": {"rz": 44.84, "xy": 43.53},
    "dram_bytes_per_cell_step": {"rz": 350.6, "xy": 345.1},
    "fp64_flops_per_cell_stage": {"rz": 1011.7, "xy": 940.4},
}
# Streaming steps (dt_h, dt_f, dt_g) of the general-face-path leg.
GEN_STEPS = (0.3, 0.4, 0.3)
METRIC = "GCUPS coupled EULBFS step, FP32 batched vs FP64 plain; p50/p99 solve latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="eulbfs", choices=["eulbfs", "reference"])
    ap.add_argument("--domains", type=int, default=64)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--tile", type=int, default=0,
                    help="rows per work item (strip segment height); 0: picked by eulbfs_autotune on the batch")
    ap.add_argument("--graph", type=int, default=16, help="steps per captured CUDA graph (0: direct launches)")
    ap.add_argument("--stage-launches", action="store_true",
                    help="one launch per Runge-Kutta stage instead of one per time step")
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--gen-steps", type=int, default=200,
                    help="steps of the general-streaming-step leg (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="seconds of oracle work per CPU-baseline leg (one thread, all cores)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", type=int, default=500, help="requests in the serving leg (0: skip)")
    ap.add_argument("--serve-fp64", type=int, default=50,
                    help="requests of the trace also served as sequential FP64 solves (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=4.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA-peak measurement")
    ap.add_argument("--geometry", default="rz", choices=["rz", "xy"],
                    help="rz: axisymmetric (r, z) droplet domains; xy: planar 2-D")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(base: int, rank: int) -> int:
    """Each rank solves its own independent batch."""
    return base + 1000 * rank


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_sources_sha256() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2507_03366_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def counters_current() -> bool:
    """The ncu counters above were taken on the kernel as it is now."""
    return kernel_sources_sha256() == COUNTERS["sources_sha256"]


def workload(n_domains: int, seed: int, geometry: str = "rz"):
    from paper_2507_03366_gb300 import workloads as wl
    return wl.static_droplet_batch(n_domains, seed=seed, axisymmetric=geometry == "rz")


def host_cores() -> dict:
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def oracle_rate(case, seconds: float, threads: int) -> dict:
    """The oracle as it stands on one domain for about `seconds` of work with
    `threads` host threads; GCUPS over the steps it finished."""
    import oracle
    used = oracle.set_threads(threads)
    s = oracle.OracleSolver(case)
    s.step(1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        s.step(2)
        steps += 2
    el = time.perf_counter() - t0
    return {"value": case.cells * steps / el / 1e9, "unit": "GCUPS", "cores": used, "steps": steps,
            "seconds": el}


def cpu_baseline(cases, seconds: float) -> dict:
    """The FP64 oracle on the smallest domain of the batch, single-threaded and
    on every host core (a partial-run rate: the oracle is a baseline, not a
    target)."""
    case = min(cases, key=lambda c: c.cells)
    one = oracle_rate(case, seconds, 1)
    allc = oracle_rate(case, seconds, os.cpu_count() or 1)
    return {"value": allc["value"], "unit": "GCUPS", "cores": allc["cores"], "kind": "oracle",
            "sample": f"{allc['steps']} steps of domain {case.name} ({case.nx}x{case.ny}) of the batch, FP64 oracle "
                      f"on {allc['cores']} host threads (OpenMP over rows and faces), {allc['seconds']:.1f} s",
            "single_thread": {"value": one["value"], "unit": "GCUPS", "cores": 1,
                              "sample": f"{one['steps']} steps of the same domain, {one['seconds']:.1f} s"},
            "host": host_cores()}


def workload_config(cases, world: int, args) -> dict:
    cells = sum(c.cells for c in cases)
    geo = "axisymmetric (r, z)" if cases and cases[0].axisymmetric else "planar 2-D"
    return {"workload": f"static droplet freezing batch, {geo}: {len(cases)} domains per GPU, sides "
                        f"{{128,192,256,384,512}}, {cells} cells per GPU",
            "global_batch": len(cases) * world, "seq_len": cells, "parallelism": f"independent domains x{world}",
            "precision": "FP32C",
            "work_item": (f"31-column strips, rows cut into runs of about {args.tile}"
                          + (" (autotuned)" if getattr(args, "autotuned", False) else ""))
            if args.tile else "31-column strip segments, height autotuned", "graph_steps": args.graph,
            "launch": ("one per Runge-Kutta stage" if args.stage_launches else
                       f"whole steps, {min(args.graph, 16)} per launch" if args.graph else
                       "whole steps, up to 16 per launch"),
            "l2": (f"working set {cells * 28 * 3 / 1e6:.0f} MB > L2 (129 MB): three 28 B/cell state buffers, "
                   "no flush needed" if cells * 28 * 3 > 129e6 else
                   f"working set {cells * 28 * 3 / 1e6:.0f} MB, not larger than L2 (129 MB)")}


def measure_fma_peaks(stream) -> dict:
    """FP32 (scalar and packed f32x2) and FP64 FMA throughput of this GPU,
    each from one launch of about 0.2 s after a short calibration launch,
    with the SM clock sampled during the launches."""
    import torch
    from paper_2507_03366_gb300 import eulbfs
    out = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for name, kind in (("fp32", eulbfs.PEAK_FP32), ("fp32x2", eulbfs.PEAK_FP32X2), ("fp64", eulbfs.PEAK_FP64)):
        probe = eulbfs.peak_fma(kind, 2000, stream)
        iters = max(2000, int(2000 * 200.0 / max(probe["ms"], 1e-3)))
        r = eulbfs.peak_fma(kind, iters, stream)
        out[name] = {"tflops": r["flops_per_s"] / 1e12, "fma_warp_inst_per_s": r["fma_warp_inst_per_s"],
                     "ms": r["ms"], "iters": iters}
    out["clocks"] = clocks.stop()
    return out


def roofline(cells, geometry, ms_per_step, launches_per_step, hbm_gbs, peaks) -> dict:
    """The stage kernel's roofs over a time step (one launch per step, or
    one per Runge-Kutta stage); the top level names the one with the largest
    fraction, which is the one the kernel meets first."""
    current = counters_current()
    s = ms_per_step * 1e-3
    hbm = {}
    for key, b, what in (("compulsory", BYTES_COMPULSORY[1], "state read and written once per step"),
                         ("stage_by_stage", BYTES_STAGE_BY_STAGE[1], "each Runge-Kutta stage's input and output")):
        ach = b * cells / s / 1e9
        hbm[key] = {"bytes_per_cell_step": b, "meaning": what, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": ach / hbm_gbs}
    dram = COUNTERS["dram_bytes_per_cell_step"][geometry] * cells if current else None
    hbm["dram_measured"] = {"bytes_per_cell_step": COUNTERS["dram_bytes_per_cell_step"][geometry] if current else None,
                            "achieved": dram / s / 1e9 if dram else None, "peak": hbm_gbs, "unit": "GB/s",
                            "frac": dram / s / 1e9 / hbm_gbs if dram else None}
    roofs = {"hbm_" + k: dict(v, bound="hbm", peak_source="measured copy bandwidth (MEASURED_PEAKS.json)")
             for k, v in hbm.items()}
    if peaks:
        fp32_peak = max(peaks["fp32"]["tflops"], peaks["fp32x2"]["tflops"])
        issue_peak = peaks["fp32"]["fma_warp_inst_per_s"]
        flops = COUNTERS["fp32_flops_per_cell_stage"][geometry] * STAGES * cells if current else None
        inst = COUNTERS["warp_inst_per_cell_stage"][geometry] * STAGES * cells if current else None
        roofs["fp32"] = {"bound": "alu", "flops_per_cell_stage": COUNTERS["fp32_flops_per_cell_stage"][geometry]
                         if current else None, "achieved": flops / s / 1e12 if flops else None, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": flops / s / 1e12 / fp32_peak if flops else None,
                         "peak_source": "measured this run: FMA-chain kernel, best of scalar and f32x2"}
        roofs["issue"] = {"bound": "alu", "warp_inst_per_cell_stage": COUNTERS["warp_inst_per_cell_stage"][geometry]
                          if current else None, "achieved": inst / s if inst else None, "peak": issue_peak,
                          "unit": "warp-inst/s", "frac": inst / s / issue_peak if inst else None,
                          "peak_source": "measured this run: warp instructions per second of the scalar FP32 "
                                         "FMA-chain kernel (one FFMA per lane per instruction)"}
    top = max((v for v in roofs.values() if v.get("frac") is not None), key=lambda v: v["frac"])
    return {"bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "traffic": dram / launches_per_step if dram else None,
            "binding_roof": next(k for k, v in roofs.items() if v is top),
            "kernel": "eulbfs::stage_kernel<float>", "launches_per_step": launches_per_step,
            "avg_launch_ms": ms_per_step / launches_per_step, "counters_current": current, "roofs": roofs}


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the machine's host cores: each step is
    a bounded sample of the workload (one domain of the batch)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cases = workload(args.domains, rank_seed(args.seed, 0), args.geometry)
    import oracle
    case = min(cases, key=lambda c: c.cells)
    cores = oracle.set_threads(os.cpu_count() or 1)
    s = oracle.OracleSolver(case)
    for _ in range(args.warmup):
        s.step(1)
    # bounded: about two minutes of oracle work for the whole timed part
    probe_t = time.perf_counter()
    s.step(2)
    per_step = (time.perf_counter() - probe_t) / 2
    steps = max(1, min(args.steps, int(120.0 / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    s.step(steps)
    el = time.perf_counter() - t0
    value = case.cells * steps / el / 1e9
    sample = (f"{steps} steps of domain {case.name} ({case.nx}x{case.ny}) of the batch, "
              f"FP64 oracle on {cores} host threads, {el:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cases, 1, args),
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(solver, stream, steps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2507_03366_gb300 import eulbfs

    cases = workload(args.domains, rank_seed(args.seed, rank), args.geometry)
    cells = sum(c.cells for c in cases)
    stream = torch.cuda.Stream()
    peaks = None if args.no_peaks else measure_fma_peaks(stream.cuda_stream)
    sol = eulbfs.Solver(cases, precision=eulbfs.FP32C, stream=stream.cuda_stream)
    tuning = None
    if args.tile == 0:
        # the autotuner times each candidate height on the live batch (its
        # steps are part of the warm-up); every solver below uses the winner
        args.tile, _ = sol.autotune(5)
        args.autotuned = True
        tuning = {str(k): v for k, v in sorted(sol.autotune_report().items())}
    sol.set_tile(args.tile)
    sol.set_whole_step(not args.stage_launches)
    if args.graph:
        sol.use_graphs(args.graph)
    for _ in range(max(3, args.warmup)):
        sol.step(1)
    if args.graph:
        sol.step(args.graph)    # the graph is captured (and replayed once) before the timed region
    sol.sync()

    # ---- device-resident timed region ----------------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = sol.launch_count()
    ev0.record(stream)
    sol.step(args.steps)
    ev1.record(stream)
    launches = sol.launch_count() - launches0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    sol.sync()   # raises on a non-finite state
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, world)
    total_cells = reduce_sum(float(cells), world)
    value = total_cells * args.steps / (ms_max * 1e-3) / 1e9

    mp = measured_peaks()
    hbm = mp["hbm_gbs"] if mp else 6800.0
    roof = roofline(cells, args.geometry, ms / args.steps, launches / args.steps, hbm, peaks)
    if not mp:
        for v in roof["roofs"].values():
            if v.get("unit") == "GB/s":
                v["peak_source"] = "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"

    # ---- FP64 plain GPU step on the same workload ------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        s64 = eulbfs.Solver(cases, precision=eulbfs.FP64, stream=stream.cuda_stream)
        s64.set_tile(args.tile)
        s64.step(2)
        s64.sync()
        ms64 = timed_steps(s64, stream, args.fp64_steps)
        fp64 = {"value": cells * args.fp64_steps / (ms64 * 1e-3) / 1e9, "unit": "GCUPS",
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps}
        if peaks and counters_current():
            # the FP64 step is bound by the FP64 pipe
            f64 = COUNTERS["fp64_flops_per_cell_stage"][args.geometry]
            ach64 = f64 * cells * STAGES * args.fp64_steps / (ms64 * 1e-3) / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach64, "peak": peaks["fp64"]["tflops"], "unit": "TFLOP/s",
                                "frac": ach64 / peaks["fp64"]["tflops"], "kernel": "eulbfs::stage_kernel<double>",
                                "flops_per_cell_stage": f64,
                                "peak_source": "measured this run: FP64 FMA-chain kernel"}
        s64.close()

    # ---- the same batch with per-distribution streaming steps (reading R26) ----
    # dt_h = dt_g = 0.3, dt_f = 0.4: every domain takes the general face path
    gen = None
    if args.gen_steps > 0:
        gcases = []
        for c in cases:
            g = copy.copy(c)
            g.dt_h, g.dt_f, g.dt_g = GEN_STEPS
            gcases.append(g)
        sg = eulbfs.Solver(gcases, precision=eulbfs.FP32C, stream=stream.cuda_stream)
        sg.set_tile(args.tile)
        sg.step(3)
        sg.sync()
        msg = timed_steps(sg, stream, args.gen_steps)
        gv = cells * args.gen_steps / (msg * 1e-3) / 1e9
        gen = {"value": gv, "unit": "GCUPS", "steps": args.gen_steps, "ms_per_step": msg / args.gen_steps,
               "dt_stream_hfg": list(GEN_STEPS),
               "relative_to_half_step_path": gv / (cells * args.steps / (ms * 1e-3) / 1e9),
               "nonfinite": any(sg.diag(k)["nonfinite"] for k in range(len(gcases)))}
        sg.close()

    # ---- end to end through the public API with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        sol.close()
        del sol
        torch.cuda.synchronize()
        pinned = []
        for c in cases:   # the caller's inputs in pinned host memory
            for k in list(c.init):
                t = torch.empty(c.init[k].shape, dtype=torch.float64, pin_memory=True)
                t.numpy()[...] = c.init[k]
                pinned.append(t)
                c.init[k] = t.numpy()
        outs = [{k: torch.empty(c.cells, dtype=torch.float64, pin_memory=True).numpy()
                 for k in ("H", "T", "Fl", "C", "p", "u", "v")} for c in cases]
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = eulbfs.Solver(cases, precision=eulbfs.FP32C, stream=stream.cuda_stream)
        s2.set_tile(args.tile)
        s2.step(args.steps)
        for k, c in enumerate(cases):
            fo = eulbfs.FieldsOut(*[eulbfs._ptr(outs[k][f]) for f in ("H", "T", "Fl", "C", "p", "u", "v")])
            eulbfs._check(eulbfs.lib().eulbfs_fields(s2._h, k, fo))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        barrier(world)
        el = reduce_max(el, world)
        s2.close()
        h2d = sum(8 * c.cells * 6 for c in cases)
        d2h = sum(8 * c.cells * 7 for c in cases)
        e2e = {"value": total_cells * args.steps / el / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "solver creation from pinned host fields, K steps, all fields back to pinned host"}

    # ---- serving: Poisson-arriving impact cases, continuous batching -----------
    serving_out = None
    if args.serve > 0:
        from paper_2507_03366_gb300 import serving
        from paper_2507_03366_gb300 import workloads as wl
        reqs = wl.impact_requests(args.serve, seed=5 + 1000 * rank, axisymmetric=args.geometry == "rz",
                                  hysteresis=True)
        budget = int(args.serve_budget_gb * 2 ** 30)
        rep = serving.serve(reqs, precision=eulbfs.FP32C, budget_bytes=budget, chunk=16,
                            stream=stream.cuda_stream, realtime=True)
        serving_out = rep.summary()
        serving_out["arrival_rate_hz"] = 20.0
        serving_out["workload"] = ("droplet impact on a cold plate, sides U[256,1024]/32, We U[10,200], "
                                   "Re U[100,2000], St U[0.05,0.5], drop released 0.1 side above the plate, end time t U/D = 0.015, "
                                   "plate angles theta_eq 82 / theta_adv 100 / theta_r 39 deg (hysteresis wall)")
        if args.serve_fp64 > 0:
            # the first requests of the same trace (same arrival times), served
            # as sequential FP64 solves (one case on the device at a time) and
            # with FP32C continuous batching
            sub = reqs[:args.serve_fp64]
            r64 = serving.serve(sub, precision=eulbfs.FP64, budget_bytes=budget, chunk=16,
                                stream=stream.cuda_stream, realtime=True, resident_cap=1)
            r32 = serving.serve(sub, precision=eulbfs.FP32C, budget_bytes=budget, chunk=16,
                                stream=stream.cuda_stream, realtime=True)
            serving_out["subset"] = {"requests": len(sub), "fp64_sequential": r64.summary(),
                                     "fp32c_batched": r32.summary()}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    cpu = None if args.no_cpu else cpu_baseline(cases, args.cpu_seconds)
    line = {
        "metric": METRIC,
        "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (H, C compensated hi/lo)", "data": "synthetic",
        "config": workload_config(cases, world, args),
        "roofline": roof,
        "peaks": peaks,
        "autotune_ms_per_step": tuning,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "fp64_plain": fp64,
        "general_streaming": gen,
        "serving": serving_out,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
