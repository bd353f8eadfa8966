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

BYTES_PER_CELL_STEP = {1: 244, 0: 352}    # algorithmic HBM bytes per cell per time step (FP32C, FP64)
STAGES = 3
# Per cell and stage of the FP32C stage kernel, from the ncu counters of one
# capture of each geometry (24 domains, 2.32 M cells, stages 0-2): FP32
# operations (FFMA counted as 2) and warp instructions issued.  They are the
# formulation's arithmetic and the kernel's instruction stream, so they change
# only with the face/cell algebra or the code.
FP32_FLOPS_PER_CELL_STAGE = {"rz": 939, "xy": 901}
WARP_INST_PER_CELL_STAGE = {"rz": 43.1, "xy": 41.7}
# DRAM bytes per cell per launch of the stage kernel (ncu, average of the 3
# stages of the same capture, scaled by cells).
DRAM_BYTES_PER_CELL_LAUNCH = 64.4
# FP64 operations per cell per stage of the FP64 stage kernel (DFMA counted as
# 2), from the ncu counters of one capture of each geometry.
FP64_FLOPS_PER_CELL_STAGE = {"rz": 1035, "xy": 958}
# Streaming steps (dt_h, dt_f, dt_g) of the general-face-path leg.
GEN_STEPS = (0.3, 0.4, 0.3)
# Peaks from unit counts: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x SM clock;
# 4 warp instructions issued per SM per clock (one per scheduler); 2 FP64
# FMA lanes per SM (ncu's sustained DFMA peak) x 2 flops x SM clock.
SMS, FP32_LANES_PER_SM, ISSUE_PER_SM_CLK, FP64_LANES_PER_SM = 152, 128, 4, 2


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
    ap.add_argument("--graph", type=int, default=0, help="steps per captured CUDA graph (0: direct launches)")
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--gen-steps", type=int, default=200,
                    help="steps of the general-streaming-step leg (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", type=int, default=500, help="requests in the serving leg (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=4.0)
    ap.add_argument("--no-cpu", action="store_true")
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
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
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


def workload(n_domains: int, seed: int, geometry: str = "rz"):
    from paper_2507_03366_gb300 import workloads as wl
    return wl.static_droplet_batch(n_domains, seed=seed, axisymmetric=geometry == "rz")


def cpu_baseline(cases, seconds: float) -> dict:
    """The oracle as it stands, single-threaded, on the first domains of the
    batch for a bounded number of steps (a partial-run rate)."""
    import oracle
    case = min(cases, key=lambda c: c.cells)
    s = oracle.OracleSolver(case)
    s.step(1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        s.step(2)
        steps += 2
    el = time.perf_counter() - t0
    return {"value": case.cells * steps / el / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of domain {case.name} ({case.nx}x{case.ny}) of the batch, "
                      f"single-threaded FP64 oracle, {el:.1f} s"}


METRIC = "GCUPS coupled EULBFS step, FP32 batched vs FP64 plain; p50/p99 solve latency"


def binding_roof(bytes_per_launch: float, flops_per_launch: float, hbm_gbs: float, fp32_tflops: float) -> str:
    """The roof that bounds a launch: the one whose minimum time (bytes over
    bandwidth, or flops over the FP32 rate) is the longer; "hbm" on a tie."""
    t_mem = bytes_per_launch / (hbm_gbs * 1e9)
    t_alu = flops_per_launch / (fp32_tflops * 1e12)
    return "hbm" if t_mem >= t_alu else "alu"


def workload_config(cases, world: int, args) -> dict:
    cells = sum(c.cells for c in cases)
    geo = "axisymmetric (r, z)" if cases and cases[0].axisymmetric else "planar 2-D"
    return {"workload": f"static droplet freezing batch, {geo}: {len(cases)} domains per GPU, sides "
                        f"{{128,192,256,384,512}}, {cells} cells per GPU",
            "global_batch": len(cases) * world, "seq_len": cells, "parallelism": f"independent domains x{world}",
            "precision": "FP32C",
            "work_item": (f"31x{args.tile} strip segment" + (" (autotuned)" if getattr(args, "autotuned", False) else ""))
            if args.tile else "31-column strip segments, height autotuned", "graph_steps": args.graph,
            "l2": (f"working set {cells * 28 * 3 / 1e6:.0f} MB > L2 (129 MB): three 28 B/cell state buffers, "
                   "no flush needed" if cells * 28 * 3 > 129e6 else
                   f"working set {cells * 28 * 3 / 1e6:.0f} MB, not larger than L2 (129 MB)")}


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the machine's host cores: each step is
    a bounded sample of the workload (one domain of the batch)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cases = workload(args.domains, rank_seed(args.seed, 0), args.geometry)
    import oracle
    case = min(cases, key=lambda c: c.cells)
    s = oracle.OracleSolver(case)
    for _ in range(args.warmup):
        s.step(1)
    # bounded: about two minutes of oracle work for the whole timed part
    steps = max(1, min(args.steps, int(120.0 * 1.2e5 / case.cells)))
    t0 = time.perf_counter()
    s.step(steps)
    el = time.perf_counter() - t0
    value = case.cells * steps / el / 1e9
    sample = (f"{steps} steps of domain {case.name} ({case.nx}x{case.ny}) of the batch, "
              f"single-threaded FP64 oracle, {el:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cases, 1, args),
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    sol = eulbfs.Solver(cases, precision=eulbfs.FP32C, stream=stream.cuda_stream)
    if args.tile == 0:
        # the autotuner times each candidate height on the live batch (its
        # steps are part of the warm-up); every solver below uses the winner
        args.tile, _ = sol.autotune(5)
        args.autotuned = True
    sol.set_tile(args.tile)
    if args.graph:
        sol.use_graphs(args.graph)
    for _ in range(max(3, args.warmup)):
        sol.step(1)
    sol.sync()

    # ---- device-resident timed region ----------------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    sol.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    sol.sync()   # raises on a non-finite state
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, world)
    total_cells = reduce_sum(float(cells), world)
    value = total_cells * args.steps / (ms_max * 1e-3) / 1e9
    launches = STAGES * args.steps

    # ---- roofline of the stage kernel (the only kernel in the region) --------
    # Arithmetic intensity ~940 flop / 81.3 B = 11.6 flop/B sits at the machine
    # balance (80.5 TFLOP/s / 6.78 TB/s = 11.9 flop/B): the binding roof is the
    # one whose minimum launch time is the longer; the other is reported beside
    # it, with the instruction-issue rate that the kernel actually meets.
    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    clk_mhz = (peaks or {}).get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * clk_mhz * 1e6 / 1e12      # TFLOP/s
    per_launch_ms = ms / launches
    alg_bytes = BYTES_PER_CELL_STEP[1] / STAGES * cells
    achieved_gbs = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    flops = FP32_FLOPS_PER_CELL_STAGE[args.geometry] * cells
    achieved_tf = flops / (per_launch_ms * 1e-3) / 1e12
    issue_peak = SMS * ISSUE_PER_SM_CLK * clk_mhz * 1e6
    issue = WARP_INST_PER_CELL_STAGE[args.geometry] * cells / (per_launch_ms * 1e-3)
    alu = {"achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved_tf / fp32_peak,
           "peak_source": "unit counts x max SM clock (152 x 128 x 2 x %.0f MHz)" % clk_mhz,
           "flops_per_launch": flops}
    mem = {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
           "peak_source": "measured" if peaks else "fallback", "algorithmic_bytes_per_launch": alg_bytes}
    hbm_bound = binding_roof(alg_bytes, flops, hbm, fp32_peak) == "hbm"
    top, other = (mem, alu) if hbm_bound else (alu, mem)
    roofline = {"bound": "hbm" if hbm_bound else "alu", **top, "traffic": DRAM_BYTES_PER_CELL_LAUNCH * cells,
                "kernel": "eulbfs::stage_kernel<float>", "avg_launch_ms": per_launch_ms,
                ("alu" if hbm_bound else "hbm"): other,
                "issue": {"achieved": issue, "peak": issue_peak, "unit": "warp-inst/s", "frac": issue / issue_peak,
                          "peak_source": "152 SMs x 4 schedulers x %.0f MHz" % clk_mhz,
                          "warp_inst_per_cell_stage": WARP_INST_PER_CELL_STAGE[args.geometry]}}

    # ---- FP64 plain GPU step on the same workload ------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        s64 = eulbfs.Solver(cases, precision=eulbfs.FP64, stream=stream.cuda_stream)
        s64.set_tile(args.tile)
        s64.step(2)
        s64.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(args.fp64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": cells * args.fp64_steps / (ms64 * 1e-3) / 1e9, "unit": "GCUPS",
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps}
        f64 = FP64_FLOPS_PER_CELL_STAGE[args.geometry]
        if f64:
            # the FP64 step is bound by the FP64 pipe (85 % busy in ncu)
            fp64_peak = SMS * FP64_LANES_PER_SM * 2 * clk_mhz * 1e6 / 1e12
            ach64 = f64 * cells * STAGES * args.fp64_steps / (ms64 * 1e-3) / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach64, "peak": fp64_peak, "unit": "TFLOP/s",
                                "frac": ach64 / fp64_peak, "kernel": "eulbfs::stage_kernel<double>",
                                "peak_source": "unit counts x max SM clock (152 x 2 x 2 x %.0f MHz)" % clk_mhz}
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
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sg.step(args.gen_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        msg = e0.elapsed_time(e1)
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
        rep = serving.serve(reqs, precision=eulbfs.FP32C, budget_bytes=int(args.serve_budget_gb * 2 ** 30),
                            chunk=16, stream=stream.cuda_stream, realtime=True)
        serving_out = rep.summary()
        serving_out["arrival_rate_hz"] = 20.0
        serving_out["workload"] = ("droplet impact on a cold plate, sides U[256,1024]/32, We U[10,200], "
                                   "Re U[100,2000], St U[0.05,0.5], drop released 0.1 side above the plate, end time t U/D = 0.015, "
                                   "plate angles theta_eq 82 / theta_adv 100 / theta_r 39 deg (hysteresis wall)")
        if fp64:
            serving_out["fp64_sequential_s_est"] = rep.cell_steps / (fp64["value"] * 1e9)

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
        "roofline": roofline,
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
