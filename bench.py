#!/usr/bin/env python
"""Benchmark of the FSM surface generator on GB300.

One step = one pass of the whole hot path over one surface: device planning
(edge, phase and path tables), the persistent tile sweep with decode and
store, the FP64 roughness moments and the profiles -- the 5x5 mm, 1 um
ball-end raster (25 Mcells, 12 passes; the metric's configuration). Prints
ONE JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (launched by torch.distributed.run) every rank predicts its own
surface (weak scaling, no collective on the data path); the time is the max
over ranks. --impl reference times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
import argparse
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

METRIC = "edge-point evals/s and surfaces/s at <=5 nm height error; p50/p99 latency"
UNIT = "cutting edge-point evaluations/s"
# algorithmic work of one cutting evaluation (the survey's count for the
# FP32 path): 9 FFMA (3x3 pose) + 3 FADD (tile offset) + 2 FMUL (bin
# scaling) = 23 flops; as instruction lanes, those 14 plus 2 float->int
# conversions, ~6 integer/compare operations, 1 shared load and at most 1
# shared atomic = 24. (The kernel's own pose is cheaper: 7 FFMA + 2 FADD in
# cell units, 16 flops.)
FP32_FLOPS_PER_EVAL = 23
ISSUE_LANES_PER_EVAL = 24
KERNEL_FLOPS_PER_EVAL = 16
FP64_HEIGHT_FLOPS = 5     # FP64 maps: the height row of the pose (2 FMA + 1 add) per evaluation
TRAJ_FP64_FLOPS = 15      # one FP64 pose: 3 x (2 FMA + 1 add)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-paper", action="store_true")
    ap.add_argument("--skip-trajectory", action="store_true")
    ap.add_argument("--skip-wall", action="store_true")
    ap.add_argument("--skip-tilted", action="store_true")
    ap.add_argument("--skip-filter", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the single-surface FP32 and FP64 steps (profiling runs)")
    ap.add_argument("--batch-size", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-seconds", type=float, default=6.0, help="seconds of arrivals per served rate")
    ap.add_argument("--serve-rates", default="40,80,160,320,640,960",
                    help="Poisson arrival rates (requests/s) of the served leg, comma separated")
    ap.add_argument("--serve-setups", type=int, default=64,
                    help="served requests draw tool and set-up from a catalogue of this many (0: all distinct)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the served leg (after the single-surface steps) and print its record")
    ap.add_argument("--width", type=float, default=5.0,
                    help="patch width in mm (5.0 = the measured configuration; smaller for profiling)")
    args = ap.parse_args()
    if args.skip_extras:
        for k in ("cpu_baseline", "batch", "large", "serve", "paper", "trajectory", "wall", "filter", "tilted"):
            setattr(args, "skip_" + k, True)
    if args.serve_only:
        for k in ("cpu_baseline", "batch", "large", "paper", "trajectory", "wall", "filter", "fp64", "tilted"):
            setattr(args, "skip_" + k, True)
    global WIDTH
    WIDTH = args.width
    return args


WIDTH = 5.0


def workload(precision):
    from paper_2603_28160_gb300 import workloads as W
    return W.raster_ball_d10(precision=precision, width=WIDTH)


def config(w, extra=None):
    p = w.process
    c = {"workload": "raster_ball_d10 (ball D=10, 4 flutes, helix 30, runout 5um@30, lead 15, 12 passes "
                     "fz=0.08 ae=0.3, 200 edge pts, 0.1 deg/step, %gx%g mm @ 1 um)" % (WIDTH, WIDTH),
         "cells": p.nx * p.ny, "passes": p.n_passes, "time_steps": p.n_passes * p.steps_per_pass,
         "trajectory_points": w.trajectory_points, "precision": p.precision,
         "l2": "flushed between timed steps (256 MB write, outside the step events)"}
    if extra:
        c.update(extra)
    return c


def src_hash():
    h = hashlib.sha256()
    for f in ("fsm_kernels.cu", "fsm_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2603_28160_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "fsm_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx.append(float(v[2]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(fraction=1.0, n_passes=4):
    """Bounded sample for the CPU oracle: the n_passes middle passes of the
    workload (same tool, grid and path), or the middle `fraction` of each of
    those passes (the spindle phase of the first sampled step kept as in the
    full path)."""
    from paper_2603_28160_gb300 import workloads as W
    w = workload("fp64")
    p = w.process
    n_passes = min(n_passes, p.n_passes)
    mid = (p.n_passes - n_passes) // 2
    p2 = p.replace(n_passes=n_passes, pass_y0=p.pass_y0 + mid * p.ae)
    if fraction < 1.0:
        n = max(1, int(p.steps_per_pass * fraction))
        start = (p.steps_per_pass - n) // 2
        s_first = mid * p.steps_per_pass + start
        fs = w.tool.n_teeth * p.fz / round(360.0 / p.rot_step_deg)
        p2 = p2.replace(steps_per_pass=n, pass_x0=p.pass_x0 + start * fs,
                        phase0_deg=(p.phase0_deg + p.rot_sense * s_first * p.rot_step_deg) % 360.0)
        return W.Workload(w.name + "_%dpasses_%.2f" % (n_passes, fraction), w.tool, p2)
    return W.Workload(w.name + "_%dpasses" % n_passes, w.tool, p2)


def run_oracle_step(sample, threads):
    from oracle import oracle as O
    t0 = time.perf_counter()
    r = O.fsm(sample, n_threads=threads)
    return time.perf_counter() - t0, r.stats


def host_cpu():
    """Host core count and CPU model string (lscpu, else /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    model = v
                    break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or platform.machine()


def cpu_baseline():
    """The oracle as it stands on the host cores: single-threaded on two
    middle passes, and on every core over all twelve passes (the time steps
    split into one contiguous range per thread, private maps merged by
    minimum). The line's value is the all-core figure."""
    nproc, model = host_cpu()
    one = oracle_sample(n_passes=2)
    dt1, st1 = run_oracle_step(one, 1)
    full = oracle_sample(n_passes=workload("fp64").process.n_passes)
    dta, sta = run_oracle_step(full, nproc)
    v1, va = st1["cutting"] / dt1, sta["cutting"] / dta
    return {"value": va, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "all 12 passes of the same workload on %d threads (%.2f s wall, %d trajectory points); "
                      "single thread: the 2 middle passes (%.2f s, %d trajectory points)"
                      % (nproc, dta, sta["trajectory_points"], dt1, st1["trajectory_points"]),
            "nproc": nproc, "cpu_model": model,
            "threads_1": {"value": v1, "unit": UNIT, "seconds": dt1, "cutting": st1["cutting"],
                          "trajectory_points": st1["trajectory_points"], "trajectory_points_per_s":
                              st1["trajectory_points"] / dt1},
            "threads_all": {"value": va, "unit": UNIT, "threads": nproc, "seconds": dta, "cutting": sta["cutting"],
                            "trajectory_points": sta["trajectory_points"], "trajectory_points_per_s":
                                sta["trajectory_points"] / dta}}


def reference_arm(args):
    """The FP64 CPU oracle as the reference arm, on every host core (bounded
    sample per step)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1 and rank != 0:
        return 0
    # a run of many steps samples the middle tenth of each of the four passes
    # (about a tenth of the time per step) so the whole run stays in minutes
    fraction = 1.0 if args.steps + args.warmup <= 40 else 0.1
    sample = oracle_sample(fraction)
    nproc, model = host_cpu()
    threads = nproc
    for _ in range(args.warmup):
        run_oracle_step(sample, threads)
    times, cut = [], 0
    for _ in range(args.steps):
        dt, st = run_oracle_step(sample, threads)
        times.append(dt)
        cut = st["cutting"]
    ms = 1e3 * sum(times) / len(times)
    value = cut / (ms / 1e3)
    what = "4 of the 12 passes of the workload per step" + ("" if fraction == 1.0 else ", the middle tenth of each pass")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config(workload("fp64"), {"sample": "4 middle passes of 12" + (
                "" if fraction == 1.0 else ", middle tenth of each"), "oracle_threads": threads}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": what,
                             "nproc": nproc, "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def unit_peaks(device):
    """Measured rates of the units the kernels are bound by (the
    micro-benchmarks of libfsm_probe.so, best of 3 x 3 runs), with the
    copy bandwidth from MEASURED_PEAKS.json for the HBM-bound kernels."""
    from paper_2603_28160_gb300 import probe
    runs = [probe.run(device, 3) for _ in range(3)]
    best = {k: max(r[k] for r in runs) for k in probe.FIELDS}
    best["source"] = "measured by libfsm_probe.so on this GPU (sustained, every SM, best of 9 runs)"
    return best


def issue_peak(sms, sm_mhz):
    """Instruction-issue peak: 4 schedulers x 32 lanes per SM per clock."""
    return sms * 128 * sm_mhz * 1e6


def sweep_roofline(cutting, atomics, sweep_ms, peaks, sms, sm_mhz):
    """The sweep against the units that bound it: FP32 arithmetic (the
    survey's 23 flops per cutting evaluation against the measured FFMA rate),
    instruction issue (24 algorithmic instruction lanes per cutting
    evaluation against 128 lanes per SM per clock at the sampled clock) and
    shared-memory atomics (the atomicMin updates against the measured
    conflict-free rate)."""
    t = sweep_ms / 1e3
    a = cutting * FP32_FLOPS_PER_EVAL / t / 1e12
    fp32 = peaks["fp32_flops"] / 1e12
    ip = issue_peak(sms, sm_mhz)
    ia = cutting * ISSUE_LANES_PER_EVAL / t
    return {"bound": "alu", "achieved": a, "peak": fp32, "unit": "TFLOP/s", "frac": a / fp32,
            "peak_source": "measured FP32 FFMA rate (libfsm_probe.so)",
            "flops_per_cutting_eval": FP32_FLOPS_PER_EVAL, "kernel_flops_per_cutting_eval": KERNEL_FLOPS_PER_EVAL,
            "issue": {"achieved": ia, "peak": ip, "unit": "instruction lanes/s", "frac": ia / ip,
                      "lanes_per_cutting_eval": ISSUE_LANES_PER_EVAL,
                      "peak_source": "%d SMs x 128 lanes x %.0f MHz (median SM clock of the timed region)"
                                     % (sms, sm_mhz)},
            "atoms": {"achieved": atomics / t, "peak": peaks["atoms32_ops"], "unit": "shared atomicMin/s",
                      "frac": atomics / t / peaks["atoms32_ops"],
                      "peak_source": "measured conflict-free 32-bit shared atomicMin rate"}}


def fp64_roofline(cutting, atomics, sweep_ms, peaks, sms, sm_mhz):
    """Roofline of an FP64-map sweep: its binning is FP32 arithmetic (as for
    FP32 maps); its heights run on the FP64 pipe, at most one 5-flop height
    per evaluation (the phase form shares one among the revolutions of a
    phase), against the measured DFMA rate."""
    r = sweep_roofline(cutting, atomics, sweep_ms, peaks, sms, sm_mhz)
    a64 = cutting * FP64_HEIGHT_FLOPS / (sweep_ms / 1e3) / 1e12
    p64 = peaks["fp64_flops"] / 1e12
    r["fp64_heights"] = {"achieved": a64, "peak": p64, "unit": "TFLOP/s (FP64)", "frac": a64 / p64,
                         "flops_per_cutting_eval": FP64_HEIGHT_FLOPS, "peak_source": "measured DFMA rate",
                         "note": "upper bound on the heights computed"}
    r["atoms"]["peak"] = peaks["atoms64_ops"]
    r["atoms"]["frac"] = r["atoms"]["achieved"] / peaks["atoms64_ops"]
    r["atoms"]["peak_source"] = "measured conflict-free 64-bit shared atomicMin rate"
    return r


def time_steps(ctx, F, tool, proc, out, rough, K, flush, precision, events_sweep=True):
    import torch
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sw = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in sw:  # create the underlying CUDA events before handing them over
        a.record(st)
        b.record(st)
    torch.cuda.synchronize()
    prec_code = F.FSM_FP64 if precision == "fp64" else F.FSM_FP32
    for i in range(K):
        flush.zero_()
        ev[i][0].record(st)
        ctx.predict_surface(tool, proc, out, events=sw[i] if events_sweep else None)
        ctx.roughness_async(out, prec_code, rough)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sweep_ms = [a.elapsed_time(b) for a, b in sw]
    return step_ms, sweep_ms


def large_grid_leg(ctx, F, flush, steps=2):
    """The 20x20 mm, 2 um flat-end floor finish (100 Mcells) in FP32: one
    surface per step (planning, sweep, roughness)."""
    import torch
    from paper_2603_28160_gb300 import workloads as W
    w = W.floor_flat_d12(precision="fp32")
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    out = F.heights_tensor(w.process)
    rough = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    ctx.predict_surface(t, p, out, counters=cnt)
    torch.cuda.synchronize()
    cutting = int(cnt[1].item())
    step_ms, sweep_ms = time_steps(ctx, F, t, p, out, rough, steps, flush, "fp32")
    ms = sum(step_ms) / len(step_ms)
    del out
    torch.cuda.empty_cache()
    return {"workload": "floor_flat_d12: flat D=12, 3 flutes 35/38/41 deg helix, runout 8 um, fz=%.4f (seeded), "
                        "7 passes ae=4.8, 300 flank + 6000 bottom pts, 0.05 deg/step, 20x20 mm @ 2 um" % w.process.fz,
            "cells": w.process.cells, "trajectory_points": w.trajectory_points, "cutting": cutting,
            "steps": steps, "ms_per_step": ms, "sweep_ms": sum(sweep_ms) / len(sweep_ms),
            "value": cutting / (ms / 1e3), "unit": UNIT, "surfaces_per_s": 1e3 / ms}


def tilted_feed_leg(ctx, F, flush, steps=3):
    """The bench's ball raster fed at 30 degrees from +X (the tool path and
    tool turned; passes enough to cross the 5 x 5 mm patch at 1 um), FP32,
    one surface per step (planning, sweep, roughness), beside the same tool
    on the +X path of the same generator."""
    import torch
    from paper_2603_28160_gb300 import workloads as W
    res = {}
    for deg in (30.0, 0.0):
        w = W.raster_ball_tilted(precision="fp32", feed_dir_deg=deg)
        t, p = ctx.tool(w.tool), ctx.process(w.process)
        out = F.heights_tensor(w.process)
        rough = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        ctx.predict_surface(t, p, out, counters=cnt)
        torch.cuda.synchronize()
        cutting, evaluated = int(cnt[1].item()), int(cnt[0].item())
        step_ms, sweep_ms = time_steps(ctx, F, t, p, out, rough, steps, flush, "fp32")
        ms = sum(step_ms) / len(step_ms)
        res["feed_%g_deg" % deg] = {"passes": w.process.n_passes, "trajectory_points": w.trajectory_points,
                                    "cutting": cutting, "evaluated": evaluated, "ms_per_step": ms,
                                    "sweep_ms": sum(sweep_ms) / len(sweep_ms), "value": cutting / (ms / 1e3),
                                    "unit": UNIT, "surfaces_per_s": 1e3 / ms}
        del out
    res["workload"] = ("raster_ball_tilted: the ball raster's tool and conditions fed at 30 deg (and 0 deg) from +X, "
                       "passes ae=0.3 crossing the 5x5 mm patch at 1 um")
    return res


def side_wall_leg(ctx, F, flush, steps=3):
    """The side of the side-plus-floor finish: the 20 x 1 mm wall at 2 um
    (5 Mcells) that the flat D=12 flank leaves on one pass, FP32, one
    surface per step (planning, sweep, roughness)."""
    import torch
    from paper_2603_28160_gb300 import workloads as W
    w = W.side_wall_flat_d12(precision="fp32")
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    out = F.heights_tensor(w.process)
    rough = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    # the library's autotuner picks the sweep shape for this workload; later
    # calls with the same shape of problem use it
    tuned = ctx.autotune(t, p, out)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    ctx.predict_surface(t, p, out, counters=cnt)
    torch.cuda.synchronize()
    cutting = int(cnt[1].item())
    step_ms, sweep_ms = time_steps(ctx, F, t, p, out, rough, steps, flush, "fp32")
    ms = sum(step_ms) / len(step_ms)
    del out
    return {"workload": "side_wall_flat_d12: flank of flat D=12, 3 flutes 35/38/41 deg, runout 8 um, radial depth "
                        "0.3, one pass, %d flank pts, 0.05 deg/step; wall map 20x1 mm @ 2 um over x and z"
                        % w.tool.n_edge,
            "cells": w.process.cells, "trajectory_points": w.trajectory_points, "cutting": cutting, "steps": steps,
            "ms_per_step": ms, "sweep_ms": sum(sweep_ms) / len(sweep_ms), "value": cutting / (ms / 1e3),
            "unit": UNIT, "surfaces_per_s": 1e3 / ms,
            "sweep_shape": {"tile": list(tuned["tile"]), "threads": tuned["threads"],
                            "ctas_per_sm": tuned["ctas_per_sm"]}}


def batched_leg(ctx, F, n, steps, peaks, rank=0, ws_count=1):
    """The Latin-hypercube batch (FP32) in one persistent launch per precision,
    prepared once and replayed as a CUDA graph. With several ranks each rank
    takes a disjoint share of the surfaces (see paper_2603_28160_gb300.shard)."""
    import torch
    from paper_2603_28160_gb300 import shard
    from paper_2603_28160_gb300 import workloads as W
    allw = W.lhs_batch(n=n)
    mine = shard.split_by_cost([w.process.cells for w in allw], ws_count)[rank]
    ws = [allw[i] for i in mine]
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    rough = torch.zeros(len(ws) * F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    counted = ctx.batch(tools, procs, outs, rough_buf=rough, counters=cnt)
    counted.run()
    torch.cuda.synchronize()
    cutting = int(cnt[1].item())
    counted.close()
    b = ctx.batch(tools, procs, outs, rough_buf=rough)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, e in ev:
        with torch.cuda.stream(s):
            a.record(s)
            g.replay()
            e.record(s)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(e) for a, e in ev]
    mean = sum(ms) / len(ms)
    cells = sum(w.process.cells for w in ws)
    # the stated comparison: the same first surfaces predicted one at a time
    # by the plain FP64 single-surface path, against the FP32 batch of them
    k = min(256, len(ws))
    sub = [W.Workload(w.name, w.tool, w.process.replace(precision="fp64")) for w in ws[:k]]
    t_sub = [ctx.tool(w.tool) for w in sub]
    p_sub = [ctx.process(w.process) for w in sub]
    o_sub = [F.heights_tensor(w.process) for w in sub]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t_, p_, o_ in zip(t_sub, p_sub, o_sub):
        ctx.predict_surface(t_, p_, o_)
        ctx.roughness_async(o_, F.FSM_FP64, rough)
    e1.record()
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    del o_sub
    b32 = ctx.batch(tools[:k], procs[:k], outs[:k], rough_buf=rough)
    b32.run()
    torch.cuda.synchronize()
    e0.record()
    b32.run()
    e1.record()
    torch.cuda.synchronize()
    fp32_ms = e0.elapsed_time(e1)
    b32.close()
    del outs
    b.close()
    torch.cuda.empty_cache()
    return {"workload": "lhs_batch: %d seeded Latin-hypercube surfaces (ball/flat, D 4-16, 2-6 flutes, helix "
                        "20-45, runout 0-15 um, lead/tilt 0-20, fz 0.03-0.2, ae 0.1-1.0, patches 0.5-4 mm "
                        "at 1-5 um), FP32, 200 edge pts, 0.1 deg/step" % n,
            "surfaces": len(ws), "cells": cells, "cutting": cutting, "steps": steps, "ms_per_step": mean,
            "surfaces_per_s": len(ws) / (mean / 1e3), "value": cutting / (mean / 1e3), "unit": UNIT,
            "launch": "prepared batch replayed as one CUDA graph (planning, persistent sweep, roughness)",
            "roofline": {"bound": "alu", "achieved": cutting * FP32_FLOPS_PER_EVAL / (mean / 1e3) / 1e12,
                         "peak": peaks["fp32_flops"] / 1e12, "unit": "TFLOP/s",
                         "frac": cutting * FP32_FLOPS_PER_EVAL / (mean / 1e3) / peaks["fp32_flops"],
                         "flops_per_cutting_eval": FP32_FLOPS_PER_EVAL,
                         "note": "whole replay time (planning, sweeps and roughness of every surface)",
                         "peak_source": "measured FP32 FFMA rate (libfsm_probe.so)"},
            "vs_plain_fp64": {"surfaces": k, "fp32_batch_surfaces_per_s": k / (fp32_ms / 1e3),
                              "fp64_single_surface_surfaces_per_s": k / (fp64_ms / 1e3),
                              "speedup": fp64_ms / fp32_ms}}


# mean optimised-FSM time per 10 x 5 mm surface over the nine conditions of
# the paper's computational-performance table (Section 4.3, its CPU)
PAPER_EFSM_S_MEAN = 0.5711
# fixed time step that reproduces that table's trajectory-point counts
PAPER_DT_S = 2e-7


def paper_case2_leg(ctx, F, flush, steps=3):
    """The paper's own performance workload: the round-insert face mill of
    Case 2 over 10 x 5 mm at 5 um, zero runout, the nine (vc, fz, ap)
    conditions of Section 4.3, in FP64 and FP32, each as one prepared batch
    of nine and one surface at a time (host enqueue included), each surface
    with its roughness."""
    import torch
    from paper_2603_28160_gb300 import workloads as W
    out = {}
    for prec in ("fp64", "fp32"):
        ws = W.paper_grid(precision=prec, dt_s=PAPER_DT_S)
        tools = [ctx.tool(w.tool) for w in ws]
        procs = [ctx.process(w.process) for w in ws]
        outs = [F.heights_tensor(w.process) for w in ws]
        rough = torch.zeros(len(ws) * F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
        # the library's autotuner picks the sweep shape on the first condition
        # (recorded in the context for the single-surface calls; passed to the
        # batch explicitly)
        tuned = ctx.autotune(tools[0], procs[0], outs[0])
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        ctx.predict_batch(tools, procs, outs, rough_buf=rough, counters=cnt, tile=tuned["tile"],
                          threads=tuned["threads"])
        torch.cuda.synchronize()
        cutting = int(cnt[1].item())
        code = F.FSM_FP64 if prec == "fp64" else F.FSM_FP32
        b = ctx.batch(tools, procs, outs, rough_buf=rough, tile=tuned["tile"], threads=tuned["threads"])

        def one_step(batched):
            if batched:
                b.run()
            else:
                for t_, p_, o_ in zip(tools, procs, outs):
                    ctx.predict_surface(t_, p_, o_)
                    ctx.roughness_async(o_, code, rough)

        def timed(batched):
            for _ in range(3):
                one_step(batched)
            torch.cuda.synchronize()
            ms = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                one_step(batched)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return sum(ms) / len(ms)
        mean = timed(True)
        single = timed(False)
        b.close()
        out[prec] = {"ms_per_9_surfaces": mean, "ms_per_surface": mean / len(ws),
                     "sweep_shape": {"tile": list(tuned["tile"]), "threads": tuned["threads"]},
                     "surfaces_per_s": len(ws) / (mean / 1e3), "cutting": cutting,
                     "value": cutting / (mean / 1e3), "unit": UNIT, "launch": "prepared batch of 9",
                     "one_at_a_time": {"ms_per_surface": single / len(ws),
                                       "launch": "fsm_predict_surface + fsm_roughness per surface, "
                                                 "host enqueue included"}}
        del outs
    torch.cuda.empty_cache()
    grid = W.paper_grid(dt_s=PAPER_DT_S)
    return {"workload": "paper Case 2 face mill (2 round inserts R=5, D=10, rake 0.6 deg), 10x5 mm @ 5 um, "
                        "zero runout, 9 (vc, fz, ap) conditions of Section 4.3, 100 edge pts, fixed 0.2 us "
                        "time step (the table's trajectory-point counts)",
            "cells_per_surface": grid[0].process.cells,
            "time_steps_total": sum(w.process.trajectory_steps for w in grid),
            "trajectory_points_total": sum(w.trajectory_points for w in grid), "steps": steps, **out,
            "paper_efsm_s_per_surface_mean": PAPER_EFSM_S_MEAN,
            "paper_note": "context only: the paper's optimised CPU FSM on its own machine and discretisation"}


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def trajectory_leg(ctx, F, flush, peaks, steps=5):
    """Trajectory map of the metric's workload (every time step of the 12
    passes, every tooth): planning, the per-phase argmin table and the
    records, timed as one call. Bound by the 32-byte record writes."""
    import torch
    w = workload("fp32")
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    raw = ctx.trajectory(t, p)
    for _ in range(3):
        ctx.trajectory(t, p, out=raw)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.trajectory(t, p, out=raw)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    mean = sum(ms) / len(ms)
    n = raw.shape[0]
    peak, src = measured_hbm_gbs()
    gbs = n * F.TRAJ_BYTES / (mean / 1e3) / 1e9
    tf = n * TRAJ_FP64_FLOPS / (mean / 1e3) / 1e12
    del raw
    # one FP64 pose per record (15 flops) against GB300's FP64 rate binds
    # before the 32 B record write does
    return {"records": n, "bytes": n * F.TRAJ_BYTES, "ms": mean, "records_per_s": n / (mean / 1e3),
            "roofline": {"bound": "alu", "achieved": tf, "peak": peaks["fp64_flops"] / 1e12,
                         "unit": "TFLOP/s (FP64)", "frac": tf / (peaks["fp64_flops"] / 1e12),
                         "peak_source": "measured DFMA rate (libfsm_probe.so)",
                         "note": "algorithmic work = 15 FP64 flops (one pose) per (step, tooth) record; call "
                                 "time includes planning and the per-phase argmin table",
                         "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                 "peak_source": src + " copy bandwidth", "bytes_per_record": F.TRAJ_BYTES}}}


def filter_leg(ctx, F, flush, steps=3):
    """The paper's measurement filters (S 10 um, L 0.8 mm) on the metric's
    25 Mcell map at 1 um, FP32 and FP64 maps."""
    import torch
    pitch, ls, lc = 0.001, 0.010, 0.8
    ts, tc = int(ls / pitch + 1e-9), int(lc / pitch + 1e-9)
    fma_per_cell = 2 * (2 * ts + 1) + 2 * (2 * tc + 1)
    out = {"lambda_s_mm": ls, "lambda_c_mm": lc, "taps_per_cell": fma_per_cell}
    for prec in ("fp32", "fp64"):
        w = workload(prec)
        H = F.heights_tensor(w.process)
        ctx.predict_surface(ctx.tool(w.tool), ctx.process(w.process), H)
        sl = torch.empty_like(H)
        for _ in range(2):
            ctx.filter(H, pitch, ls, lc, out=sl)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.filter(H, pitch, ls, lc, out=sl)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        mean = sum(ms) / len(ms)
        cells = H.numel()
        tflops = 2.0 * fma_per_cell * cells / (mean / 1e3) / 1e12
        out[prec] = {"ms": mean, "cells_per_s": cells / (mean / 1e3),
                     "achieved_tflops": tflops,
                     "arith": "FP32" if prec == "fp32" else "double-float on the FP32 pipes (~11 FP32 ops per tap)"}
        del H, sl
    torch.cuda.empty_cache()
    return out


def busy_fraction(log):
    """Share of the span of a batch log during which some batch was on the
    device (union of the batches' device-time intervals)."""
    iv = sorted((b["t_start_ms"], b["t_end_ms"]) for b in log)
    if not iv:
        return None
    busy, cur_s, cur_e = 0.0, iv[0][0], iv[0][1]
    for a, b in iv[1:]:
        if a > cur_e:
            busy += cur_e - cur_s
            cur_s, cur_e = a, b
        else:
            cur_e = max(cur_e, b)
    busy += cur_e - cur_s
    span = iv[-1][1] - iv[0][0]
    return busy / span if span > 0 else None


def served_run(ctx, F, seconds, rate, setups, seed=5):
    """One Poisson request stream through fsm_submit/fsm_poll (continuous
    batching, 120 GB admission budget, 70 % FP32 / 30 % FP64, 0.25-25 Mcells),
    every result polled and released in arrival order."""
    import threading
    from paper_2603_28160_gb300 import workloads as W
    n = max(1, int(seconds * rate))
    reqs = W.serve_stream(n, seed=seed, n_setups=setups or None)
    arrivals = W.poisson_arrivals(n, rate, seed=seed)
    handles = [(ctx.tool(w.tool), ctx.process(w.process)) for w in reqs]
    ctx.server_start(budget_bytes=120 << 30, n_streams=4, max_batch=64)
    tickets = [None] * n
    lat, queue = [0.0] * n, [0.0] * n
    done = threading.Event()

    def collect():
        for i in range(n):
            while tickets[i] is None:
                time.sleep(0.0005)
            r = ctx.poll(tickets[i], timeout_ms=-1)
            lat[i], queue[i] = r["latency_s"], r["queue_s"]
            ctx.release(tickets[i])
        done.set()

    try:
        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for i in range(n):
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets[i] = ctx.submit(*handles[i])
        done.wait()
        elapsed = time.perf_counter() - t0
        th.join()
        stats = ctx.server_stats()
        log = ctx.server_batches()
    finally:
        ctx.server_stop()
    srt = sorted(lat)
    return {"rate": rate, "requests": n, "fp64_requests": sum(w.process.precision == "fp64" for w in reqs),
            "cells": sum(w.process.cells for w in reqs), "elapsed_s": elapsed, "surfaces_per_s": n / elapsed,
            "cells_per_s": sum(w.process.cells for w in reqs) / elapsed,
            "p50_ms": 1e3 * srt[len(srt) // 2], "p99_ms": 1e3 * srt[min(n - 1, int(0.99 * n))],
            "queue_p50_ms": 1e3 * sorted(queue)[n // 2], "queue_p99_ms": 1e3 * sorted(queue)[min(n - 1, int(0.99 * n))],
            "batches": stats["batches"], "mean_batch": n / max(1, stats["batches"]),
            "table_hits": stats["table_hits"], "table_misses": stats["table_misses"],
            "bytes_peak_gb": stats["bytes_peak"] / 2 ** 30, "queue_peak": stats["queue_peak"],
            "device_busy": busy_fraction(log)}


def served_leg(ctx, F, seconds, rates, setups, seed=5):
    """Served stream at increasing Poisson rates: throughput tracks the
    arrivals until the server saturates; the highest throughput reached is
    its capacity on this request mix."""
    import torch
    from paper_2603_28160_gb300 import workloads as W
    runs = [served_run(ctx, F, seconds, r, setups, seed) for r in rates]
    best = max(runs, key=lambda r: r["surfaces_per_s"])
    # the plain FP64 single-surface form on the same requests (the first 64
    # of the stream, all in FP64, one fsm_predict_surface + fsm_roughness at a
    # time), for the served-versus-plain comparison
    k = 64
    sub = [W.Workload(w.name, w.tool, w.process.replace(precision="fp64"))
           for w in W.serve_stream(k, seed=seed, n_setups=setups or None)]
    rough = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    hs = [(ctx.tool(w.tool), ctx.process(w.process)) for w in sub]
    out = torch.empty(max(w.process.cells for w in sub), dtype=torch.float64, device="cuda")
    for (t_, p_), w in list(zip(hs, sub))[:2]:  # warm
        ctx.predict_surface(t_, p_, out[:w.process.cells])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for (t_, p_), w in zip(hs, sub):
        o_ = out[:w.process.cells].view(w.process.ny, w.process.nx)
        ctx.predict_surface(t_, p_, o_)
        ctx.roughness_async(o_, F.FSM_FP64, rough)
    e1.record()
    torch.cuda.synchronize()
    plain = k / (e0.elapsed_time(e1) / 1e3)
    del out
    torch.cuda.empty_cache()
    sat = [r for r in runs if r["surfaces_per_s"] < 0.9 * r["rate"]]
    return {"workload": "serve_stream: Poisson arrivals, batch-distribution requests (%s), 0.25-25 Mcells, "
                        "30%% FP64, %g s per rate" % ("tools and set-ups from a catalogue of %d" % setups if setups
                                                     else "every tool and set-up drawn afresh", seconds),
            "budget_gb": 120, "streams": 4, "max_batch": 64, "rates": runs,
            "capacity_surfaces_per_s": best["surfaces_per_s"], "capacity_at_rate": best["rate"],
            "saturated": bool(sat), "saturation_rate": sat[0]["rate"] if sat else None,
            "surfaces_per_s": best["surfaces_per_s"], "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"],
            "vs_plain_fp64": {"fp64_single_surface_surfaces_per_s": plain, "requests": k,
                              "served_capacity_over_plain_fp64": best["surfaces_per_s"] / plain,
                              "note": "the first %d requests of the stream in FP64, one surface at a time" % k}}


def gb300_arm(args):
    import torch

    from paper_2603_28160_gb300 import fsm as F

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    ctx = F.Context(local)
    w = workload(args.precision)
    tool, proc = ctx.tool(w.tool), ctx.process(w.process)
    out = F.heights_tensor(w.process)
    rough = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    prec_code = F.FSM_FP64 if args.precision == "fp64" else F.FSM_FP32

    # work counts of one step (deterministic), outside the timed region
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    ctx.predict_surface(tool, proc, out, counters=cnt)
    torch.cuda.synchronize()
    evaluated, cutting, rebinned, atomics = [int(x) for x in cnt.cpu()]

    for _ in range(args.warmup):
        ctx.predict_surface(tool, proc, out)
        ctx.roughness_async(out, prec_code, rough)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    step_ms, sweep_ms = time_steps(ctx, F, tool, proc, out, rough, args.steps, flush, args.precision)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(ws)
    clk = clocks.stop()
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, ws)
    value = ws * cutting / (ms / 1e3)
    p50 = statistics.median(step_ms)
    p99 = sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]
    sweep_mean = sum(sweep_ms) / len(sweep_ms)
    # the measured rates of the units the kernels are bound by (outside the
    # timed region) and the clock the timed region ran at
    peaks = unit_peaks(local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz_live = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0

    # end to end through the C ABI with host buffers: descriptors cross the
    # ABI and the map plus the roughness record are copied back to pinned
    # host memory every step. Two streams with a buffer set each, so the
    # copies of step i overlap the compute of step i+1; every copy has
    # completed when the timed region ends. Each step starts with an L2 flush
    # on its stream, inside the wall clock (so no step finds the previous
    # one's map in L2; the figure includes the flushes' time).
    nbuf = 2
    streams = [torch.cuda.Stream() for _ in range(nbuf)]
    flushes = [flush] + [torch.empty_like(flush) for _ in range(nbuf - 1)]
    outs = [out] + [torch.empty_like(out) for _ in range(nbuf - 1)]
    roughs = [rough] + [torch.zeros_like(rough) for _ in range(nbuf - 1)]
    host_maps = [torch.empty(out.shape, dtype=out.dtype, pin_memory=True) for _ in range(nbuf)]
    host_roughs = [torch.empty(F.ROUGH_BYTES, dtype=torch.uint8, pin_memory=True) for _ in range(nbuf)]

    def e2e_step(i):
        k = i % nbuf
        st = streams[k]
        with torch.cuda.stream(st):
            flushes[k].zero_()
            t_ = ctx.tool(w.tool)
            p_ = ctx.process(w.process)
            ctx.predict_surface(t_, p_, outs[k], stream=st)
            ctx.roughness_async(outs[k], prec_code, roughs[k], stream=st)
            host_maps[k].copy_(outs[k], non_blocking=True)
            host_roughs[k].copy_(roughs[k], non_blocking=True)

    e2e_steps = max(6, args.steps // 2)
    for i in range(2 * nbuf):
        e2e_step(i)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
    d2h = out.numel() * out.element_size() + F.ROUGH_BYTES
    h2d = F.C.sizeof(F.ToolDesc) + F.C.sizeof(F.ProcessDesc)

    # the plain FP64 single-surface form, for comparison
    fp64 = None
    if not args.skip_fp64 and args.precision != "fp64":
        w64 = workload("fp64")
        t64, p64 = ctx.tool(w64.tool), ctx.process(w64.process)
        out64 = F.heights_tensor(w64.process)
        cnt64 = torch.zeros(4, dtype=torch.int64, device="cuda")
        ctx.predict_surface(t64, p64, out64, counters=cnt64)
        torch.cuda.synchronize()
        cut64 = int(cnt64[1].item())
        at64 = int(cnt64[3].item())
        k64 = max(3, args.steps // 10)
        s64, sw64 = time_steps(ctx, F, t64, p64, out64, rough, k64, flush, "fp64")
        ms64 = max_over_ranks(sum(s64) / len(s64), ws)
        sw64_mean = sum(sw64) / len(sw64)
        fp64 = {"value": ws * cut64 / (ms64 / 1e3), "ms_per_step": ms64, "steps": k64,
                "sweep_ms": sw64_mean, "cutting": cut64,
                "roofline": fp64_roofline(cut64, at64, sw64_mean, peaks, sms, sm_mhz_live)}
        del out64

    large = None
    if not args.skip_large and rank == 0:
        large = large_grid_leg(ctx, F, flush)
    filt = None
    if not args.skip_filter and rank == 0:
        filt = filter_leg(ctx, F, flush)
    side = None
    if not args.skip_wall and rank == 0:
        side = side_wall_leg(ctx, F, flush)
    tilted = None
    if not args.skip_tilted and rank == 0:
        tilted = tilted_feed_leg(ctx, F, flush)
    traj = None
    if not args.skip_trajectory and rank == 0:
        traj = trajectory_leg(ctx, F, flush, peaks)
    paper = None
    if not args.skip_paper and rank == 0:
        paper = paper_case2_leg(ctx, F, flush)
    batched = None
    if not args.skip_batch:
        batched = batched_leg(ctx, F, args.batch_size, args.batch_steps, peaks, rank, ws)
        if ws > 1:
            bms = max_over_ranks(batched["ms_per_step"], ws)
            batched["ms_per_step_max_over_ranks"] = bms
            batched["surfaces_per_s"] = args.batch_size / (bms / 1e3)
    served = None
    if not args.skip_serve and rank == 0:
        served = served_leg(ctx, F, args.serve_seconds, [float(r) for r in args.serve_rates.split(",")],
                            args.serve_setups)
    barrier(ws)

    if rank != 0:
        return 0

    # roofline of the dominant kernel (the sweep): algorithmic work per
    # cutting evaluation / live event time of the sweep launch, against the
    # measured unit rates
    roof = (sweep_roofline if args.precision == "fp32" else fp64_roofline)(cutting, atomics, sweep_mean, peaks, sms,
                                                                           sm_mhz_live)
    traffic = None
    prof = os.path.join(ROOT, "profiles", "sweep_%s_raster_ball_d10.json" % args.precision)
    if os.path.exists(prof):
        try:
            pj = json.load(open(prof))
            if pj.get("src_hash") == src_hash():
                traffic = pj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    roof.update({"traffic": traffic, "kernel": "sweep_kernel<%s>" % args.precision.upper(), "sweep_ms": sweep_mean})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": config(w, {"parallelism": "replicas" if ws > 1 else "single GPU"}),
        "surfaces_per_s": ws / (ms / 1e3),
        "latency_ms": {"p50": p50, "p99": p99, "of": "single-surface steps (events, stream-ordered)"},
        "work": {"cutting": cutting, "evaluated": evaluated, "rebinned_fp64": rebinned, "atomics": atomics,
                 "trajectory_points": w.trajectory_points,
                 "trajectory_points_per_s": ws * w.trajectory_points / (ms / 1e3)},
        "roofline": roof,
        "unit_peaks": peaks,
        "e2e": {"value": ws * cutting / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3,
                "steps": e2e_steps, "streams": nbuf,
                "note": "host descriptors by value through the C ABI every step; height map and roughness copied "
                        "to pinned host memory every step, overlapping the next step's compute on a second "
                        "stream; a 256 MB L2 flush starts every step inside the wall clock; wall clock over all "
                        "steps until the last copy completes"},
        "gpu_launches": 6 * args.steps,  # plan, plan_finish, sweep, roughness setup, two moment passes
        "clocks": clk,
        "wall_s": wall,
        "fp64_single_surface": fp64,
        "large_grid": large,
        "paper_case2": paper,
        "trajectory": traj,
        "side_wall": side,
        "tilted_feed": tilted,
        "iso_filter": filt,
        "batched": batched,
        "served": served,
        "src_hash": src_hash(),
    }
    if ws == 1 and not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())
