#!/usr/bin/env python3
"""Throughput of the implicit multigroup source-term update on GB300.

One step = one update call over the whole synthetic grid (all steps of the
method: load, group table, inner Newton with the arrowhead elimination,
write-back, flux and momentum update, outer iteration, store).  The headline
form is the one the metric names: the mixed-precision solver started from the
learned warm start (``rhd_source_update_warm``: network inference on the
tensor cores, then the FP32 and FP64 passes); the surrogate is trained before
the timed region on cells of the same distribution (other seeds) that the
plain FP64 solver has advanced.  The plain FP64 Newton form (the comparison),
the mixed form without the surrogate and the FP64 form with it are timed
beside it on the same grid.
The grid is restored from a pristine device copy before every step, outside
the timed region; that copy (2 x 35 GB at the default size) also flushes L2.
The metric is cell-group source updates per second: cells x groups advanced
per second, every cell converged to the same tolerance.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                    [--workload full_256cube_ng64] [--impl ours|reference]

Under torchrun (N > 1) every rank draws its own grid (seed + rank) and the
ranks share no data: weak scaling, no collective on the data path.  Rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-group source updates/sec, mixed+surrogate vs FP64 Newton, same tol"
UNIT = "cell-group updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the plain FP64 form timed beside a mixed run (0: skip)")
    ap.add_argument("--workload", default="full_256cube_ng64")
    ap.add_argument("--n-cells", type=int, default=None, help="override the cell count")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cell-per-thread", action="store_true",
                    help="one cell per thread in every pass (the mapping whose operation "
                         "counts define the algorithmic flops; slower at 33-128 groups)")
    ap.add_argument("--lanes16", action="store_true",
                    help="33..64 groups: 16 lanes per cell in the mixed form's warp kernels "
                         "(RHD_LANES_16) instead of 32")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="time the solver from the cold start (no learned warm start)")
    ap.add_argument("--sur-train-cells", type=int, default=1 << 21)
    ap.add_argument("--sur-epochs", type=int, default=4)
    ap.add_argument("--cpu-sample", type=int, default=6144,
                    help="cells of the workload the CPU oracle baseline solves (about 15 s on "
                         "16 cores at 64 groups)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, ws: int, op: str) -> float:
    """x reduced over the ranks (max or sum); a host scalar on every rank."""
    if ws == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def allmax(x: float, ws: int) -> float:
    return _reduce(x, ws, "max")


def allsum(x: float, ws: int) -> float:
    return _reduce(x, ws, "sum")


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp_peaks() -> dict:
    """Measured scalar FMA peaks (TFLOP/s) from the fp_peak microbenchmark."""
    from paper_2407_18304_gb300 import build
    try:
        exe = build.build_fp_peak()
        out = subprocess.run([exe, "5"], capture_output=True, text=True, timeout=120, check=True)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the bench still reports, with the nominal figure
        return {"error": str(e)}


# The roofline's numerator: algorithmic operations of a call = the events the
# kernels report (rhd_events_start/stop: inner evaluations, outer passes,
# coupled residuals and Newton steps, ...) times the operations per event and
# cell-group of the counting model (oracle/opcount.py, a plain statement of the
# method's steps; its table is tests/golden/opcounts.json, regenerated by
# python -m oracle.opcount), the special functions weighted by their measured
# issue cost (fp_peak).  The kernels' own instruction streams do not enter.
OPCOUNTS = os.path.join(ROOT, "tests", "golden", "opcounts.json")
# events of each kind of launch (the names of rhd.EVENT_NAMES and of the table)
KERNEL_EVENTS = {"fp32_passes": ("eval32", "outer32"),
                 "refine": ("residdf", "stepdf"),
                 "correction": ("resid64", "step32", "finish64"),
                 "fp64_passes": ("eval64", "cached64", "outer64")}
# the per-update setup (tau_g and its reciprocals) once per cell of these counters
KERNEL_CELLS = {"correction": "cellsc", "fp64_passes": "cells64"}
# DRAM bytes (read + write) per cell-group of one launch of the dominant kernel,
# ncu on a 65536-cell sample of the same workload
# (profiles/correct_warp_kernel_65536cells_ng64.md); None once the kernel changed
DOMINANT_TRAFFIC_PER_CG = {("full_256cube_ng64", "correction"): 87.9}


def op_slots(counts: dict, weights: dict) -> float:
    """Issue slots of a tally {kind: n}: add, mul, fma and compares one each,
    div / sqrt / exp the measured multiple of an FMA."""
    return sum(v * (weights.get(k, 1.0) if k in ("div", "sqrt", "exp") else 1.0)
               for k, v in counts.items())


def algorithmic_ops(workload: str, events: dict, G: int, peaks: dict) -> dict:
    """{kernel: {"f64": slots, "f32": slots}} of the algorithm for the events counted
    (float-float operations as the FP32 operations they are made of)."""
    with open(OPCOUNTS) as f:
        full = json.load(f)
    table = full["events"].get(workload)
    if table is None:
        return {}
    w64 = peaks.get("fp64_op_slots", {})
    w32 = peaks.get("fp32_op_slots", {})
    dfc = full.get("df_fp32_ops", {})

    def df_as_f32(counts: dict) -> dict:
        out = {}
        for kind, n in counts.items():
            for k, v in dfc.get(kind, {}).items():
                out[k] = out.get(k, 0.0) + n * v
        return out

    out = {}
    for kern, evs in KERNEL_EVENTS.items():
        f64 = f32 = 0.0
        for e in evs:
            f64 += events.get(e, 0) * G * op_slots(table[e]["f64"], w64)
            f32 += events.get(e, 0) * G * op_slots(table[e]["f32"], w32)
            f32 += events.get(e, 0) * G * op_slots(df_as_f32(table[e].get("df", {})), w32)
        if kern in KERNEL_CELLS:
            f64 += events.get(KERNEL_CELLS[kern], 0) * G * op_slots(table["setup64"]["f64"], w64)
        out[kern] = {"f64": f64, "f32": f32}
    return out


def train_surrogate(args, w, dev, rank):
    """The learned warm start for this workload: training cells drawn like the
    grid (same groups, law and distributions, other seeds), advanced by the
    plain FP64 solver, then Adam (untimed setup)."""
    from paper_2407_18304_gb300 import rhd, surrogate, synth
    side, G, vmax, taumax, kind = synth.PRESETS[args.workload]
    t0 = time.perf_counter()
    sur = rhd.Surrogate(w.n_groups, 1 + rank)
    x, y = surrogate.training_set(sur, args.sur_train_cells, w.edges, w.law, v_max=vmax,
                                  tau_max=taumax, seed=9_000_000 + 1000 * rank, device=dev)
    losses = surrogate.train(sur, x, y, epochs=args.sur_epochs, batch=8192, seed=rank)
    del x, y
    torch.cuda.synchronize()
    info = {"train_cells": args.sur_train_cells, "epochs": args.sur_epochs,
            "epoch_losses": [round(v, 5) for v in losses],
            "setup_s": time.perf_counter() - t0, "tensor_core_error": sur.error_flag()}
    return sur, info


def run_ours(args, ws, rank):
    from paper_2407_18304_gb300 import rhd, synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    name = args.workload
    seed = synth.PRESET_SEED[name] + 1000 * rank
    w = synth.preset(name, device=dev, n_cells=args.n_cells, seed=seed)
    n, G = w.n_cells, w.n_groups
    prec = rhd.FP64 if args.precision == "fp64" else rhd.MIXED
    use_sur = not args.no_surrogate
    sur, sur_info = train_surrogate(args, w, dev, rank) if use_sur else (None, None)
    pristine = w.state
    st = synth.clone_state(pristine)
    status = torch.empty(n, dtype=torch.uint8, device=dev)
    iters = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def restore():
        for k in ("mom", "egas", "erad", "frad"):
            st[k].copy_(pristine[k])

    flags = (rhd.CELL_PER_THREAD if args.cell_per_thread else 0) | (
        rhd.LANES_16 if args.lanes16 else 0)

    def call(p, warm):
        args_ = dict(dt=w.dt, c_v=w.c_v, consts=w.consts, precision=p, status=status,
                     iters=iters, stream=stream, flags=flags)
        if warm:
            sur.source_update(st, w.edges, w.law, **args_)
        else:
            rhd.source_update(st, w.edges, w.law, **args_)

    def timed(p, warm, steps, warmup, sample_clocks=False):
        """warmup + steps solves; per-step CUDA-event times and outcome."""
        for _ in range(warmup):
            restore()
            call(p, warm)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        clocks = ClockSampler(dev.index)
        if sample_clocks:
            clocks.start()
        barrier(ws)
        torch.cuda.synchronize()
        if sample_clocks:
            rhd.profile_start()  # events around each launch of each call
        t0 = time.perf_counter()
        for k in range(steps):
            restore()
            starts[k].record(stream)
            if k == 0:  # marks one timed step for profilers (ncu --nvtx-include)
                torch.cuda.nvtx.range_push("rhd_step_" + ("mixed" if p == rhd.MIXED else "fp64")
                                           + ("_surrogate" if warm else ""))
            call(p, warm)
            if k == 0:
                torch.cuda.nvtx.range_pop()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        wall = time.perf_counter() - t0
        clk = clocks.stop() if sample_clocks else None
        if sample_clocks:
            rhd.profile_stop()  # per kind: rhd.profile_kernel
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        stat = status.cpu().numpy()
        it = iters.cpu().numpy().astype(np.int64)
        outcome = {"converged_fraction": float((stat <= 1).mean()),
                   "fallback_fraction": float((stat == 1).mean()),
                   "mean_newton_iters": float(it.mean())}
        return ms, wall, clk, outcome

    def side(p, warm, steps):
        ms_, _, _, out = timed(p, warm, steps, 1)
        t = allmax(sum(ms_) / 1e3, ws)
        d = {"value": allsum(float(n) * G * steps, ws) / t, "ms_per_step": 1e3 * t / steps,
             "steps": steps}
        d.update(out)
        return d

    ms, wall, clk, outcome = timed(prec, use_sur, args.steps, args.warmup, True)
    t_dev = sum(ms) / 1e3
    t_max = allmax(t_dev, ws)
    units = float(n) * G * args.steps
    total_units = allsum(units, ws)
    # FP64 form: the FP64 passes; mixed form: FP32 passes, first correction step,
    # correction, FP64 passes (no correction past 128 groups); + the inference
    launches = (1 if prec == rhd.FP64 else (4 if G <= 128 else 2)) + (1 if use_sur else 0)
    form = ("mixed" if prec == rhd.MIXED else "fp64") + ("+surrogate" if use_sur else "")

    res = {"metric": METRIC, "value": total_units / t_max, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == rhd.FP64 else ("f32+f64+bf16" if use_sur else "f32+f64"),
           "data": "synthetic (seeded generators of paper_2407_18304_gb300.synth)",
           "config": {"workload": name, "cells": n, "n_groups": G, "form": form,
                      "mapping": ("cell per thread" if args.cell_per_thread else
                                  "16 lanes per cell" if args.lanes16 else "warp per cell"),
                      "precision": args.precision, "tol": 1e-11, "tol_outer": 1e-13,
                      "l2": "state restored from a pristine copy before each step (2x state > L2)",
                      "parallelism": f"weak x{ws}, no collective"},
           "gpu_launches": args.steps * launches, "wall_s_timed": wall, "clocks": clk}
    res.update(outcome)
    if sur_info is not None:
        res["surrogate"] = sur_info

    # the comparison forms on the same grid, same tolerance
    if args.fp64_steps > 0:
        res["fp64_form"] = side(rhd.FP64, False, args.fp64_steps)
        res["speedup_vs_fp64_form"] = res["value"] / res["fp64_form"]["value"]
        if use_sur and prec == rhd.MIXED:
            res["mixed_form"] = side(rhd.MIXED, False, args.fp64_steps)
            res["fp64_surrogate_form"] = side(rhd.FP64, True, args.fp64_steps)

    # ---- roofline: algorithmic operations of the call (counting model x the
    # events the kernels report in one untimed counted call) against the
    # measured FP64 / FP32 issue rates and HBM bandwidth
    peaks = fp_peaks()
    res["fp_peaks_measured"] = peaks
    restore()
    torch.cuda.synchronize()
    rhd.events_start()
    call(prec, use_sur)
    events = rhd.events_stop()
    res["events_per_cell"] = {k: v / n for k, v in events.items() if v}
    ops = algorithmic_ops(name, events, G, peaks)
    mean_call_s = t_dev / args.steps
    bytes_alg = n * (G * 64 + 82)  # in+out FP64 SoA per call: E_g, F_g and the per-cell fields
    hbm = _measured_hbm()
    p64 = (peaks.get("fp64_fma_tflops") or 1.25) * 1e12 / 2.0  # FMA issue slots / s
    p32 = (peaks.get("fp32_fma_tflops") or 78.0) * 1e12 / 2.0
    kinds = {kname: rhd.profile_kernel(k) for k, kname in enumerate(rhd.KERNEL_NAMES)}
    kern_s = {k: v[1] / 1e3 / max(1, v[0]) for k, v in kinds.items() if v[0] > 0}
    res["kernel_ms_per_call"] = {k: 1e3 * v for k, v in kern_s.items()}
    if ops and kern_s:
        dom = max(kern_s, key=kern_s.get)
        o = ops.get(dom, {"f64": 0.0, "f32": 0.0})
        t = kern_s[dom]
        ach64, ach32 = o["f64"] / t / 1e9, o["f32"] / t / 1e9
        tr = DOMINANT_TRAFFIC_PER_CG.get((name, dom))
        tot64 = sum(v["f64"] for v in ops.values())
        tot32 = sum(v["f32"] for v in ops.values())
        t_roof = {"hbm": bytes_alg / (hbm * 1e9), "fp64": tot64 / p64, "fp32": tot32 / p32}
        res["roofline"] = {
            "bound": "alu", "achieved": ach64, "peak": p64 / 1e9, "unit": "G FP64 slots/s",
            "frac": ach64 / (p64 / 1e9),
            "traffic": tr * n * G if tr is not None else None,
            "kernel": dom, "kernel_ms": 1e3 * t,
            "what": ("algorithmic FP64 operations of the kernel per launch (counting model "
                     "tests/golden/opcounts.json x the events the kernel reports; div, sqrt and "
                     "exp at their measured issue cost) / its CUDA-event duration, against the "
                     "measured FP64 FMA issue rate (fp_peak, of measured)"),
            "fp64_slots_per_cell_group": o["f64"] / (n * G),
            "fp32": {"achieved": ach32, "peak": p32 / 1e9, "unit": "G FP32 slots/s",
                     "frac": ach32 / (p32 / 1e9), "slots_per_cell_group": o["f32"] / (n * G)},
            "hbm": {"achieved": bytes_alg / t / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": bytes_alg / t / 1e9 / hbm},
            "call": {"ms": 1e3 * mean_call_s,
                     "roofline_ms": {k: 1e3 * v for k, v in t_roof.items()},
                     "frac": max(t_roof.values()) / mean_call_s,
                     "fp64_slots_per_cell_group": tot64 / (n * G),
                     "fp32_slots_per_cell_group": tot32 / (n * G),
                     "hbm_frac": t_roof["hbm"] / mean_call_s}}
    else:
        ach = bytes_alg / mean_call_s / 1e9
        res["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                           "frac": ach / hbm, "traffic": None,
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs"}

    if not args.no_e2e:
        res["e2e"] = run_e2e(args, w, prec, dev, ws, sur)
    if rank == 0 and ws == 1:
        res["cpu_baseline"] = cpu_baseline(args, w)
    return res


BATCHED = "batched_64grids"


def run_batched(args, ws, rank):
    """64 uneven grids (16^3..96^3 cells, N_g in {4,..,64}, own opacity law
    each) advanced by one rhd_source_update_batched call per step (persistent
    launch, device work queue, replayed CUDA graph, autotuned shape); the same
    grids one rhd_source_update call each are timed beside it."""
    from paper_2407_18304_gb300 import rhd, synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    seed = 1000 * (18304 + 2) + 1000 * rank
    grids = synth.batched_grids(64, seed=seed, device=dev)
    prec = rhd.FP64 if args.precision == "fp64" else rhd.MIXED
    pristine = [synth.clone_state(g.state) for g in grids]
    units1 = float(sum(g.n_cells * g.n_groups for g in grids))
    stream = torch.cuda.current_stream()
    ctx = rhd.Context()
    specs = [rhd.GridSpec(g.state, g.edges, g.law, dt=g.dt, c_v=g.c_v, consts=g.consts,
                          precision=prec) for g in grids]

    def restore():
        for g, p in zip(grids, pristine):
            for k in ("mom", "egas", "erad", "frad"):
                g.state[k].copy_(p[k])

    def batched():
        ctx.update(specs, stream=stream)

    def per_grid():
        for g in grids:
            rhd.source_update(g.state, g.edges, g.law, dt=g.dt, c_v=g.c_v, consts=g.consts,
                              precision=prec, stream=stream)

    def timed(f, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            restore()
            f()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        clocks = ClockSampler(dev.index)
        if sample_clocks:
            clocks.start()
        barrier(ws)
        torch.cuda.synchronize()
        for a, b in ev:
            restore()
            a.record(stream)
            f()
            b.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        clk = clocks.stop() if sample_clocks else None
        return [a.elapsed_time(b) for a, b in ev], clk

    restore()
    shape = ctx.autotune(specs, stream=stream)  # untimed; leaves the state unchanged
    buckets = sorted({0 if g.n_groups <= 16 else 1 if g.n_groups <= 32 else 2 for g in grids})
    # per step: the table kernel, then per bucket its FP32 passes, first
    # correction step, correction and FP64 passes (mixed form) or its FP64 passes
    launches = 1 + len(buckets) * (4 if prec == rhd.MIXED else 1)
    ms, clk = timed(batched, args.steps, args.warmup, True)
    t_max = allmax(sum(ms) / 1e3, ws)
    total = allsum(units1 * args.steps, ws)
    res = {"metric": METRIC, "value": total / t_max, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == rhd.FP64 else "f32+f64",
           "data": "synthetic (seeded generators of paper_2407_18304_gb300.synth)",
           "config": {"workload": BATCHED, "grids": len(grids),
                      "cells": int(sum(g.n_cells for g in grids)), "cell_groups": int(units1),
                      "precision": args.precision, "tol": 1e-11, "tol_outer": 1e-13,
                      "shape": {"threads": shape[0], "cells_per_item": shape[1]},
                      "mappings": {f"bucket{b}": {"passes": ctx.mapping(b)[0],
                                                  "correction": ctx.mapping(b)[1]}
                                   for b in buckets},
                      "l2": "state restored from a pristine copy before each step (2x state > L2)",
                      "parallelism": f"weak x{ws}, no collective"},
           "gpu_launches": args.steps * launches, "clocks": clk}
    pg, _ = timed(per_grid, max(1, args.fp64_steps), 1)
    t_pg = allmax(sum(pg) / 1e3, ws)
    res["per_grid_form"] = {"value": allsum(units1 * len(pg), ws) / t_pg,
                            "ms_per_step": 1e3 * t_pg / len(pg)}
    res["speedup_vs_per_grid"] = res["value"] / res["per_grid_form"]["value"]
    bytes_alg = float(sum(g.n_cells * (g.n_groups * 64 + 82) for g in grids))
    mean_s = sum(ms) / 1e3 / args.steps
    peak = _measured_hbm()
    res["roofline"] = {"bound": "hbm", "achieved": bytes_alg / mean_s / 1e9, "peak": peak,
                       "unit": "GB/s", "frac": bytes_alg / mean_s / 1e9 / peak, "traffic": None,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                       "note": "algorithmic in+out bytes; the solve is FP64-issue bound"}
    res["e2e"] = None
    if rank == 0 and ws == 1:
        res["cpu_baseline"] = cpu_baseline(args, grids[0])
    return res


def _measured_hbm() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def run_e2e(args, w, prec, dev, ws, sur=None):
    """The same metric through the C ABI with the state in pinned host memory:
    rhd_source_update_host streams the grid through the GPU in chunks (copy
    in, solve, copy out, the copies overlapped with the solve), so every
    step's host->device inputs and device->host results are inside the timing.
    The host state is restored from a pristine pinned copy between steps,
    outside the timing."""
    from paper_2407_18304_gb300 import rhd
    n, G = w.n_cells, w.n_groups
    keys_in = ["rho", "mom", "egas", "kappa0", "erad", "frad"]
    keys_out = ["mom", "egas", "erad", "frad"]
    host = {k: torch.empty(tuple(w.state[k].shape), dtype=torch.float64, pin_memory=True)
            for k in keys_in}
    for k in keys_in:
        host[k].copy_(w.state[k])
    host["src"] = None
    pristine = {k: host[k].clone() for k in keys_out}
    host_status = torch.empty(n, dtype=torch.uint8).pin_memory()
    h2d = sum(host[k].numel() * 8 for k in keys_in)
    d2h = sum(host[k].numel() * 8 for k in keys_out) + n

    def step():
        rhd.source_update_host(host, w.edges, w.law, dt=w.dt, c_v=w.c_v, consts=w.consts,
                               precision=prec, status=host_status, surrogate=sur)

    def restore():
        for k in keys_out:
            host[k].copy_(pristine[k])

    step()  # warm-up: staging buffers, workspace
    total = 0.0
    for _ in range(args.e2e_steps):
        restore()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
    dt = allmax(total, ws)
    units = allsum(float(n) * G * args.e2e_steps, ws)
    del host, pristine
    return {"value": units / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
            "path": ("rhd_source_update_host" + (" with the learned warm start" if sur is not None
                                                 else "")
                     + ": pinned host state, 2^20-cell chunks, copies overlapped with the solve")}


def cpu_baseline(args, w):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import oracle as O
    from paper_2407_18304_gb300 import synth
    m = min(args.cpu_sample, w.n_cells)
    idx = torch.arange(m, device=w.state["rho"].device)
    sub = synth.to_numpy(synth.take_cells(w.state, idx))
    km, al = O.group_table(w.edges, O.PPL_FIXED, w.law.nu_break, w.law.seg_logk, w.law.seg_beta,
                           w.law.nu_ref)
    p = O.Params(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"],
                 h=w.consts["h"], k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt, max_iter=200)
    t0 = time.perf_counter()
    out = O.source_update(sub, p, O.Groups(w.edges, km, al))
    dt = time.perf_counter() - t0
    return {"value": m * w.n_groups / dt, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"first {m} cells of the workload, all {w.n_groups} groups, one call",
            "seconds": dt, "converged_fraction": float((out["status"] == 0).mean())}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle on the host cores, on bounded samples."""
    if rank != 0:
        return None
    import oracle as O
    from paper_2407_18304_gb300 import synth
    m = min(args.cpu_sample // 12, 512)
    if args.workload == BATCHED:
        g = synth.batched_grids(1, seed=1000 * (18304 + 2), max_side=16)[0]
        m = min(m, g.n_cells)
        w = synth.Workload(g.name, synth.take_cells(g.state, slice(0, m)), g.edges, g.law)
    else:
        w = synth.preset(args.workload, n_cells=m)
    km, al = O.group_table(w.edges, O.PPL_FIXED, w.law.nu_break, w.law.seg_logk, w.law.seg_beta,
                           w.law.nu_ref)
    p = O.Params(c=w.consts["c"], c_hat=w.consts["c_hat"], a_rad=w.consts["a_rad"],
                 h=w.consts["h"], k_B=w.consts["k_B"], c_v=w.c_v, dt=w.dt, max_iter=200)
    g = O.Groups(w.edges, km, al)
    st = synth.to_numpy(w.state)
    for _ in range(args.warmup):
        O.source_update(st, p, g)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.source_update(st, p, g)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    v = m * w.n_groups * args.steps / t
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "cells_per_step": m, "n_groups": w.n_groups},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": O.max_threads(),
                             "sample": f"{m} cells of the workload per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank = dist_setup(args) if args.impl == "ours" else (int(os.environ.get("WORLD_SIZE", "1")),
                                                             int(os.environ.get("RANK", "0")))
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    elif args.workload == BATCHED:
        res = run_batched(args, ws, rank)
    else:
        res = run_ours(args, ws, rank)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
