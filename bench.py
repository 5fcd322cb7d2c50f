#!/usr/bin/env python3
"""Throughput benchmark of the stereo surface-normal chain on GB300.

Workload: 2048x1024 driving-like scenes (ground plane, two facades, 20 boxes;
f = 2260 px, B = 0.21 m, sigma = 0.3 px, 8 % invalid), FP32 disparity, the
plain chain: range-gated 5x5 denoise, star-fill covered-depth support
(8 directions x 10 steps, k = 0.1), two-pass affine fit and normal, point
cloud, 4-connected min-index components.  One step = sn_run_frame over a
batch of frames already resident in HBM.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on the host cores, on the same workload (a band of rows per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "driving_2048x1024"
METRIC = "MPix/s (2048x1024 stereo normals chain)"
# algorithmic bytes per pixel of each launch of sn_run_frame (compulsory
# reads and writes of that kernel)
ALGO_BYTES = {
    "frame": 4 + 12 + 12 + 1,             # disp in; normals, points, mask out
    "ccl_local": 4 + 4,                   # disparity in, tile-local labels out
    "ccl_merge": 0,                       # tile borders only
    "ccl_flatten": 4 + 4,                 # labels in and out
}
FRAME_ALGO_BYTES = 33                      # disp 4 + normals 12 + points 12 + labels 4 + mask 1
# Algorithmic operations per pixel of the fused frame kernel for the default
# method, counted once per visited sample from the method's definition (not
# from this implementation's instructions): ingest 5; range-gated 5x5
# denoise 25 samples x 11 (validity and range test 2, 6 moment and 3 data
# sums) + 30 (3x3 solve) = 305; star-fill M = 8, s = 10 walks its 68 distinct
# samples once, and each visit carries the stop test and the fit's sums over
# the same support: 68 x 8 (one integer multiply-compare, 5 moment adds, 2
# data FMAs) = 544; 2x2 solve, normal and point 40.  Total 894; the kernel
# issues about 1,350 thread instructions per pixel, so this count is below
# what it executes.  Used only for the secondary (issue) roofline: the
# headline roofline of every kernel is its algorithmic bytes against HBM.
ALGO_OPS_PER_PX = {"frame": 894}
LANES_PER_SM = 128   # 4 schedulers x 32 lanes: one instruction per lane per clock
EDGE_BAND = 7        # ground-truth error is also reported within this many px of a surface edge (the widest window's radius)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=16, help="frames per step")
    ap.add_argument("--streams", type=int, default=4, help="CUDA streams the frames of a step are spread over")
    ap.add_argument("--distinct", type=int, default=8, help="distinct input frames")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-resolution batch")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--only-headline", action="store_true",
                    help="time the headline chain only (no other forms, comparators, stage calls, scene errors, "
                         "mixed batch, end to end, CPU baseline or serving): short runs for profilers")
    ap.add_argument("--scene", default=WORKLOAD,
                    help="the headline chain's scene (profiling another config, e.g. mixed_1482x994); the line "
                         "then names it in its config")
    ap.add_argument("--params", default="",
                    help="sn_params overrides of the headline pipeline, e.g. support=0,r_affine=4 or learned=1 "
                         "(for profiling another form; the line then names them in its config)")
    args = ap.parse_args()
    if args.only_headline:
        args.no_mixed = args.no_e2e = args.no_cpu_baseline = args.no_serving = True
    return args


def parse_params(text):
    """'k=v,k=v' -> dict of sn_params overrides (ints, or floats where the value has a '.')."""
    out = {}
    for item in filter(None, text.split(",")):
        k, v = item.split("=")
        out[k.strip()] = float(v) if "." in v else int(v)
    return out


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        props = torch.cuda.get_device_properties(device_index)
        uuid = str(getattr(props, "uuid", "") or "")
        if uuid:
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    return ids[device_index] if device_index < len(ids) else str(device_index)


# ---------------------------------------------------------------- helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def make_inputs(n_distinct: int, rank: int, scene: str = WORKLOAD):
    """The seeded scenes of one rank: replicas take disjoint frame numbers."""
    from scenes import make_scene
    return [make_scene(scene, frame=rank * n_distinct + i) for i in range(n_distinct)]


def max_over_ranks(x: float, dist) -> float:
    """The largest value of x over the ranks (the job ends with its slowest
    rank); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix(world: int, px_per_rank: int, ms: float) -> float:
    """Whole-job throughput: the pixels every rank processed over the slowest
    rank's time."""
    return world * px_per_rank / (ms / 1e3) / 1e6


def cpu_baseline(scenes, seconds: float):
    """The FP64 oracle as it stands on whole frames of the same workload: on
    all host cores until `seconds` of work have been spent, then on one core
    for a quarter of that (a bounded sample of whole frames)."""
    import oracle
    cores = os.cpu_count() or 1

    def timed(threads, budget):
        used = oracle.set_threads(threads)
        px, n = 0, 0
        t0 = time.perf_counter()
        while True:
            s = scenes[n % len(scenes)]
            oracle.run_frame(s.disp, s.camera)
            px += s.W * s.H
            n += 1
            if time.perf_counter() - t0 >= budget:
                break
        dt = time.perf_counter() - t0
        return px / dt / 1e6, used, n, dt

    oracle.build()
    v, used, n, dt = timed(cores, seconds)
    v1, _, n1, dt1 = timed(1, seconds / 4)
    oracle.set_threads(cores)
    return {"value": v, "unit": "MPix/s", "cores": used, "kind": "oracle",
            "sample": f"{n} whole {WORKLOAD} frames (FP32 input, full chain), {dt:.1f} s",
            "single_thread": {"value": v1, "unit": "MPix/s", "cores": 1,
                              "sample": f"{n1} whole frames, {dt1:.1f} s"},
            "per_config": oracle_per_config(cores),
            "host": f"{cores} cores, {os.uname().machine}, {cpu_model()}"}


def oracle_per_config(cores, reps=5):
    """The oracle's full chain on one frame of each of the three plain
    scenes (320x240, 1482x994, 2048x1024): median of `reps` runs on all
    host cores and on one core (ms per frame and MPix/s)."""
    import oracle
    from scenes import make_scene
    out = {}
    for name in ("planes_320x240", "mixed_1482x994", WORKLOAD):
        s = make_scene(name, frame=0)
        row = {}
        for threads in (cores, 1):
            oracle.set_threads(threads)
            ts = []
            for _ in range(reps if threads > 1 or s.W * s.H < 10 ** 6 else 1):
                t0 = time.perf_counter()
                oracle.run_frame(s.disp, s.camera)
                ts.append(time.perf_counter() - t0)
            ms = 1e3 * float(np.median(ts))
            row["all_cores" if threads > 1 else "one_core"] = {"ms": ms, "mpix_s": s.W * s.H / ms / 1e3,
                                                              "runs": len(ts)}
        out[name] = row
    oracle.set_threads(cores)
    return out


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}


def cpu_model():
    """The host CPU's model name (x86) or Arm core part."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    v = line.split(":", 1)[1].strip()
                    return ARM_PARTS.get(v.lower(), v)
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from scenes import make_scene
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    oracle.build()
    s = make_scene(WORKLOAD, frame=0)
    band = 128
    H = s.H
    bands = [s.disp[y:y + band] for y in range(0, H, band)]

    def step(i):
        b = bands[i % len(bands)]
        oracle.run_frame(b, s.camera)
        return b.shape[0] * b.shape[1]
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    px = sum(step(i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = px / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MPix/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: FP64 CPU oracle, one 2048x{band} band of the frame per step"},
        "cpu_baseline": {"value": v, "unit": "MPix/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle", "sample": f"{args.steps} bands of {band} rows"},
        "e2e": {"value": v, "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_15121_gb300 import Pipeline, sn

    scenes = make_inputs(args.distinct, rank, args.scene)
    s0 = scenes[0]
    W, H, cam = s0.W, s0.H, s0.camera
    overrides = parse_params(args.params)
    pipe = Pipeline(cam, W, H, **overrides)
    u16_in = overrides.get("in_dtype") == sn.SN_IN_U16X256
    disp = [pipe.upload(s.disp_u16 if u16_in else s.disp) for s in scenes]
    F = args.frames
    outs = [pipe.buffers() for _ in range(F)]
    stream = torch.cuda.current_stream()
    step = batch_step(pipe, disp, outs, args.streams)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sn.sn_check_device(pipe.ctx)

    # ---- timed region (device time, CUDA events on the stream every step
    # joins); no per-launch events inside it
    launches0 = sn.sn_launch_count(pipe.ctx)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id_for(dev)) as clocks:
        barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for _ in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = sn.sn_launch_count(pipe.ctx) - launches0
    elapsed_ms = t_start.elapsed_time(t_end)
    sn.sn_check_device(pipe.ctx)

    # ---- per-launch times: the same workload once more on one stream with a
    # CUDA event after every launch (kernel durations, frame latencies)
    stage_ms, nframes, frame_ms_serial = profiled_pass(pipe, disp, outs, max(1, args.steps // 4))
    frame_ms = latency_pass(pipe, disp, outs, max(1, args.steps // 4) * F)
    sn.sn_check_device(pipe.ctx)
    elapsed_ms = max_over_ranks(elapsed_ms, dist)
    value = whole_job_mpix(world, args.steps * F * W * H, elapsed_ms)

    # ---- roofline of the dominant kernel (live event times of the timed
    # region's workload): algorithmic bytes against the measured HBM peak;
    # the whole chain's bytes over the timed region beside it; the issue
    # roofline (algorithmic operations against one instruction per lane per
    # clock at the sampled SM clock, SM count from the device) is secondary
    peaks, peak_kind = load_peaks()
    avg = {k: v / max(nframes, 1) for k, v in stage_ms.items()}
    dom = max(avg, key=avg.get)
    hbm_achieved = ALGO_BYTES[dom] * W * H / (avg[dom] / 1e3) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    chain_gbs = FRAME_ALGO_BYTES * W * H / (elapsed_ms / 1e3 / (args.steps * F)) / 1e9
    traffic = load_traffic(dom)
    clk = clocks.summary()
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * LANES_PER_SM * sm_mhz * 1e6 / 1e12           # T ops/s
    alu_achieved = ALGO_OPS_PER_PX.get(dom, 0) * W * H / (avg[dom] / 1e3) / 1e12

    gt_plain = gt_error_deg(outs, scenes)

    # ---- other forms on the same scenes: uint16 (256 d) in and snorm16
    # normals out (precision form); the learned gate with FP32 and with the
    # precision form's I/O
    u16 = dict(in_dtype=sn.SN_IN_U16X256, normal_fmt=sn.SN_NORMALS_SNORM16X4)
    forms = None if args.only_headline else {
        "precision_u16_snorm16": time_form(scenes, args, u16, lambda s: s.disp_u16, 27, dist, world, hbm_peak),
        "learned_f32": time_form(scenes, args, dict(learned=1), lambda s: s.disp, FRAME_ALGO_BYTES, dist, world, hbm_peak),
        "learned_u16_snorm16": time_form(scenes, args, dict(u16, learned=1), lambda s: s.disp_u16, 27, dist,
                                         world, hbm_peak),
        # the paper's larger adaptive setting (Table perf-disc2): star-fill CD with 16 directions, 30 steps
        "cd_s30_d16_f32": time_form(scenes, args, dict(dirs=16, steps=30), lambda s: s.disp, FRAME_ALGO_BYTES,
                                    dist, world, hbm_peak),
        # star-fill with the depth-edge stop (ST s10 d8 t0.1, Table perf-disc)
        "st_s10_d8_f32": time_form(scenes, args, dict(support=2, st_t=0.1), lambda s: s.disp, FRAME_ALGO_BYTES,
                                   dist, world, hbm_peak),
        # fixed 9x9 affine window (the paper's n x n setting, n = 9)
        "fixed_9x9_f32": time_form(scenes, args, dict(support=0, r_affine=4), lambda s: s.disp, FRAME_ALGO_BYTES,
                                   dist, world, hbm_peak),
    }
    for f in (forms or {}).values():
        f["vs_plain"] = f["value"] / value
    # accuracy against throughput: plain settings of the support (the paper's
    # star-fill sizes and fixed windows) on the same scenes, and the learned
    # form against the fastest of them that is at least as accurate
    frontier = None if args.only_headline else accuracy_frontier(scenes, args, dist, world, hbm_peak, value,
                                                                 gt_plain, forms)
    # the comparison estimators of Sec. IV on the same scenes (normals only)
    comparators = None
    if world == 1 and not args.only_headline:
        comparators = {"cross": time_comparator(scenes, args, "cross", 0, world),
                       "pca_9x9": time_comparator(scenes, args, "pca", 4, world)}
    stage_calls = time_stage_calls(scenes, args) if world == 1 and not args.only_headline else None
    # every method's ground-truth error on the box-and-curve scene (1482x994)
    errors_mixed = scene_errors("mixed_1482x994") if world == 1 and not args.only_headline else None
    # the same frontier on the box-and-curve scene (the paper's box scenes),
    # where depth edges rather than far-range noise decide the error
    frontier_mixed = (scene_frontier("mixed_1482x994", args, hbm_peak)
                      if world == 1 and not args.only_headline else None)
    # mixed-resolution batch of 64 frames, one graph launch per step
    mixed = run_mixed_batch(args) if world == 1 and not args.no_mixed else None

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(pipe, scenes, args, world, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scenes, args.cpu_seconds)

    serving = None
    if world == 1 and not args.no_serving:
        serving = run_serving(args)

    if rank == 0:
        fm = sorted(frame_ms)
        pct = lambda q: fm[min(len(fm) - 1, int(round(q * (len(fm) - 1))))] if fm else None
        line = {
            "metric": METRIC, "value": value, "unit": "MPix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": f"{args.scene}: plain chain, FP32 disparity in, FP32 normals/points out, "
                            f"star-fill CD s10 d8 k0.1, 5x5 denoise; {F} frames per step "
                            f"({args.distinct} distinct seeded scenes) spread over {args.streams} CUDA streams",
                "frames_per_step": F, "W": W, "H": H, "streams": args.streams,
                "l2": "inputs+outputs per step "
                      f"{F * W * H * (4 + FRAME_ALGO_BYTES - 4) / 1e9:.2f} GB >> 129 MB L2 (no flush needed)",
                "parallelism": f"replicas x{world}",
                **({"params": overrides} if overrides else {}),
            },
            "frame_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": fm[-1] if fm else None,
                         "source": "CUDA events around each sn_run_frame on one stream, frames back to back, "
                                   "after the timed region (component passes on the forked side stream)",
                         "serialised_p50": sorted(frame_ms_serial)[len(frame_ms_serial) // 2] if frame_ms_serial else None},
            "stage_ms_per_frame": {k: round(v, 5) for k, v in avg.items()},
            "gt_error_deg": gt_plain,
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_achieved / hbm_peak,
                         "traffic": traffic["bytes_per_launch"] if traffic else None,
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback",
                         "algo_bytes_per_px": ALGO_BYTES[dom],
                         "kernel_time_source": "CUDA events after each launch, single-stream profiled pass of the "
                                               "same workload after the timed region",
                         "traffic_source": traffic["source"] if traffic else
                         "null: no ncu DRAM capture of the current build of this kernel",
                         "chain": {"achieved": chain_gbs, "frac": chain_gbs / hbm_peak,
                                   "algo_bytes_per_px": FRAME_ALGO_BYTES,
                                   "time_source": "timed region (all launches of sn_run_frame)"},
                         "issue": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Top/s",
                                   "frac": alu_achieved / alu_peak, "algo_ops_per_px": ALGO_OPS_PER_PX.get(dom),
                                   "peak_kind": f"derived: {sm_count} SMs (device) x {LANES_PER_SM} lanes x "
                                                f"{sm_mhz:.0f} MHz (median sampled SM clock)"}},
            "gpu_launches": int(launches),
            "forms": forms,
            "accuracy_frontier": frontier,
            "accuracy_frontier_mixed_1482x994": frontier_mixed,
            "comparators": comparators,
            "stage_calls": stage_calls,
            "gt_error_by_method_mixed_1482x994": errors_mixed,
            "mixed_batch": mixed,
            "clocks": clk,
            "e2e": e2e,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    pipe.close()
    if dist is not None:
        dist.destroy_process_group()


def batch_step(pipe, disp, outs, n_streams):
    """One step: every frame of the batch through sn_run_frame, frame f on
    stream f % n_streams (frames are independent; the latency-bound component
    passes of one frame overlap the next frame's frame kernel).  The current
    stream forks to the work streams and joins them again."""
    import torch
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]

    def step():
        ev = main.record_event()
        for st in streams:
            st.wait_event(ev)
        for f in range(len(outs)):
            pipe.run_frame(disp[f % len(disp)], outs[f], stream=streams[f % n_streams], write_den=False)
        for st in streams:
            main.wait_stream(st)
    return step


def profiled_pass(pipe, disp, outs, steps):
    """Stage times (ms summed per stage), frame count and per-frame times
    of `steps` passes over the batch on one stream with profiling on."""
    import torch
    from paper_2504_15121_gb300 import sn
    stream = torch.cuda.current_stream()
    sn.sn_set_profiling(pipe.ctx, True)
    sn.sn_stage_times(pipe.ctx)
    for _ in range(steps):
        for f in range(len(outs)):
            pipe.run_frame(disp[f % len(disp)], outs[f], stream=stream, write_den=False)
    torch.cuda.synchronize()
    stage_ms, nframes, frame_ms = sn.sn_stage_times(pipe.ctx, cap=steps * len(outs))
    sn.sn_set_profiling(pipe.ctx, False)
    sn.sn_check_device(pipe.ctx)
    return stage_ms, nframes, frame_ms


def latency_pass(pipe, disp, outs, n):
    """Per-frame latency as a caller sees it: CUDA events on one stream
    around each of n sn_run_frame calls (profiling off, so the component
    passes run on the forked side stream), frames back to back.  Sorted ms."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for i, (a, b) in enumerate(ev):
        a.record(stream)
        pipe.run_frame(disp[i % len(disp)], outs[i % len(outs)], stream=stream, write_den=False)
        b.record(stream)
    torch.cuda.synchronize()
    return sorted(a.elapsed_time(b) for a, b in ev)


def time_form(scenes, args, params, pick, bytes_per_px, dist, world, hbm_peak=None):
    """Device throughput and per-frame times of another form of the chain on
    the same scenes (same frames per step and step count)."""
    import torch
    from paper_2504_15121_gb300 import Pipeline, sn
    s0 = scenes[0]
    pipe = Pipeline(s0.camera, s0.W, s0.H, **params)
    disp = [pipe.upload(pick(s)) for s in scenes]
    F = args.frames
    outs = [pipe.buffers() for _ in range(F)]
    stream = torch.cuda.current_stream()
    step = batch_step(pipe, disp, outs, args.streams)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    t0.record(stream)
    steps = min(40, max(10, args.steps // 4))  # bounded: the slowest settings run at ~1.6 GPix/s
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    sn.sn_check_device(pipe.ctx)
    fm = latency_pass(pipe, disp, outs, max(1, steps // 4) * F)
    sn.sn_check_device(pipe.ctx)
    # the form's frame kernel(s) alone: live event times on one stream,
    # algorithmic bytes (the chain's less the labels) against the HBM peak
    stage_ms, nframes, _ = profiled_pass(pipe, disp, outs, max(1, steps // 8))
    gt = gt_error_deg(outs, scenes)
    pipe.close()
    ms = max_over_ranks(ms, dist)
    W, H = s0.W, s0.H
    kern_us = 1e3 * stage_ms.get("frame", 0.0) / max(nframes, 1)
    kern_gbs = (bytes_per_px - 4) * W * H / (kern_us / 1e6) / 1e9 if kern_us > 0 else None
    return {"value": whole_job_mpix(world, steps * F * W * H, ms), "unit": "MPix/s", "steps": steps,
            "frame_ms_p50": fm[len(fm) // 2] if fm else None,
            "frame_ms_p99": fm[min(len(fm) - 1, int(0.99 * (len(fm) - 1) + 0.5))] if fm else None,
            "frame_kernel_us": kern_us,
            "frame_kernel_hbm_frac": kern_gbs / hbm_peak if kern_gbs and hbm_peak else None,
            "algo_bytes_per_px": bytes_per_px,
            "gt_error_deg": gt,
            "params": {k: (v if isinstance(v, float) else int(v)) for k, v in params.items()}}


FRONTIER = {
    "cd_s20_d8": dict(dirs=8, steps=20),
    "cd_s30_d8": dict(dirs=8, steps=30),
    "cd_s10_d16": dict(dirs=16, steps=10),
    "cd_s20_d16": dict(dirs=16, steps=20),
    "fixed_5x5": dict(support=0, r_affine=2),
    "fixed_7x7": dict(support=0, r_affine=3),
    "fixed_11x11": dict(support=0, r_affine=5),
    "fixed_13x13": dict(support=0, r_affine=6),
    "fixed_15x15": dict(support=0, r_affine=7),
}


def accuracy_frontier(scenes, args, dist, world, hbm_peak, plain_value, gt_plain, forms):
    """MPix/s and mean ground-truth error of plain settings beside the default
    (CD s10 d8) and the forms already timed (CD s30 d16, fixed 9x9), and the
    learned forms' throughput against the fastest plain setting whose error
    is no worse than theirs (the comparison at equal angular error)."""
    pts = {"cd_s10_d8": frontier_point(plain_value, gt_plain)}
    for k in ("cd_s30_d16_f32", "fixed_9x9_f32", "st_s10_d8_f32"):
        pts[k[:-4]] = frontier_point(forms[k]["value"], forms[k]["gt_error_deg"])
    for name, params in FRONTIER.items():
        f = time_form(scenes, args, params, lambda s: s.disp, FRAME_ALGO_BYTES, dist, world, hbm_peak)
        pts[name] = frontier_point(f["value"], f["gt_error_deg"])
    out = {"plain": pts, "rule": FRONTIER_RULE}
    for lk in ("learned_f32", "learned_u16_snorm16"):
        f = forms[lk]
        fp = frontier_point(f["value"], f["gt_error_deg"])
        out[lk] = compare_at_equal_error(pts, fp["value"], fp["gt_error_deg"], fp["pixels"], fp["edge_band_error_deg"])
        out[lk]["elsewhere_error_deg"] = fp["elsewhere_error_deg"]
        out[lk]["vs_default_plain"] = f["value"] / plain_value
    return out


def frontier_point(value, gt):
    """One setting on the frontier: MPix/s, mean error, normals counted, and
    the mean error near surface edges and elsewhere."""
    return {"value": value, "gt_error_deg": gt["mean"], "pixels": gt["pixels"],
            "edge_band_error_deg": gt.get(f"mean_within_{EDGE_BAND}px_of_a_surface_edge"),
            "elsewhere_error_deg": gt.get("mean_elsewhere")}


FRONTIER_RULE = ("a plain setting counts as at least as accurate when its mean error is no higher and it gives "
                 "normals at no fewer than 99 % of the learned form's pixels (ST, which drops most pixels of the "
                 "driving scene as edges, does not qualify); 'also near edges' adds: and its mean error within "
                 f"{EDGE_BAND} px of a surface edge is no higher")


def scene_frontier(scene_name, args, hbm_peak, n_distinct=4):
    """accuracy_frontier on another scene: every plain setting (the default
    CD s10 d8, CD s30 d16, ST s10 d8, fixed 9x9 and FRONTIER) and the learned
    form timed on n_distinct seeded frames of it, errors against its ground
    truth, and the learned form against the fastest plain setting as accurate."""
    from scenes import make_scene
    scenes = [make_scene(scene_name, frame=300 + i) for i in range(n_distinct)]
    settings = {"cd_s10_d8": {}, "cd_s30_d16": dict(dirs=16, steps=30), "st_s10_d8": dict(support=2, st_t=0.1),
                "fixed_9x9": dict(support=0, r_affine=4), **FRONTIER}
    pts = {}
    for name, params in settings.items():
        f = time_form(scenes, args, params, lambda s: s.disp, FRAME_ALGO_BYTES, None, 1, hbm_peak)
        pts[name] = frontier_point(f["value"], f["gt_error_deg"])
    lf = time_form(scenes, args, dict(learned=1), lambda s: s.disp, FRAME_ALGO_BYTES, None, 1, hbm_peak)
    fp = frontier_point(lf["value"], lf["gt_error_deg"])
    out = {"scene": scene_name, "frames": n_distinct, "plain": pts, "rule": FRONTIER_RULE,
           "learned_f32": compare_at_equal_error(pts, fp["value"], fp["gt_error_deg"], fp["pixels"],
                                                 fp["edge_band_error_deg"])}
    out["learned_f32"]["elsewhere_error_deg"] = fp["elsewhere_error_deg"]
    out["learned_f32"]["vs_default_plain"] = lf["value"] / pts["cd_s10_d8"]["value"]
    return out


def compare_at_equal_error(plain, value, err, pixels, edge_err=None):
    """The learned form (value MPix/s, mean error err over `pixels` normals,
    mean error edge_err near surface edges) against the fastest plain
    setting at least as accurate (FRONTIER_RULE), and against the fastest
    one at least as accurate both overall and near edges."""
    ok = {k: p for k, p in plain.items() if p["gt_error_deg"] <= err and p["pixels"] >= 0.99 * pixels}
    best = max(ok, key=lambda k: ok[k]["value"]) if ok else None
    out = {"value": value, "gt_error_deg": err, "fastest_plain_as_accurate": best,
           "vs_that_plain": value / ok[best]["value"] if best else None}
    if edge_err is not None:
        ok2 = {k: p for k, p in ok.items()
               if p.get("edge_band_error_deg") is not None and p["edge_band_error_deg"] <= edge_err}
        best2 = max(ok2, key=lambda k: ok2[k]["value"]) if ok2 else None
        out.update({"edge_band_error_deg": edge_err, "fastest_plain_as_accurate_also_near_edges": best2,
                    "vs_that_plain_also_near_edges": value / ok2[best2]["value"] if best2 else None})
    return out


def time_comparator(scenes, args, which, r, world):
    """Device throughput and ground-truth error of a comparison estimator of
    Sec. IV (sn_cross_normals, sn_pca_normals) on the same scenes: normals and
    mask only, so compare it with the chain's normal stage, not the chain."""
    import torch
    from paper_2504_15121_gb300 import sn
    s0 = scenes[0]
    ctx = sn.sn_create(s0.camera, s0.W, s0.H, sn.default_params())
    try:
        disp = []
        for s in scenes:
            t = sn.empty_image(s0.H, s0.W, torch.float32)
            t.copy_(torch.from_numpy(s.disp))
            disp.append(t)
        F = args.frames
        outs = [(sn.empty_planes(3, s0.H, s0.W), sn.empty_image(s0.H, s0.W, torch.uint8)) for _ in range(F)]
        main = torch.cuda.current_stream()
        streams = [torch.cuda.Stream() for _ in range(args.streams)]

        def step():
            ev = main.record_event()
            for st in streams:
                st.wait_event(ev)
            for f in range(F):
                n, m = outs[f]
                st = streams[f % len(streams)]
                if which == "cross":
                    sn.sn_cross_normals(ctx, disp[f % len(disp)], n, m, stream=st)
                else:
                    sn.sn_pca_normals(ctx, disp[f % len(disp)], r, n, m, stream=st)
            for st in streams:
                main.wait_stream(st)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(3, args.steps // 4)
        t0.record(main)
        for _ in range(steps):
            step()
        t1.record(main)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        sn.sn_check_device(ctx)

        class _O:
            pass
        wrapped = []
        for n, m in outs[:len(scenes)]:
            o = _O()
            o.normals, o.mask = n, m
            wrapped.append(o)
        gt = gt_error_deg(wrapped, scenes)
    finally:
        sn.sn_destroy(ctx)
    return {"value": world * steps * F * s0.W * s0.H / (ms / 1e3) / 1e6, "unit": "MPix/s",
            "what": "normals + mask only", "gt_error_deg": gt}


def scene_errors(scene_name, n_frames=4):
    """Mean angular error against the generator's ground truth of every
    method on frames of one scene (Table scene-errors of the paper compares
    the adaptive, fixed-window, PCA and Cross estimators on box scenes):
    star-fill CD s10 d8 and s30 d16, ST s10 d8, the fixed 9x9 window, the
    learned form, PCA 9x9 and Cross; each frame run once on the GPU."""
    import torch
    from scenes import make_scene
    from paper_2504_15121_gb300 import Pipeline, sn
    scenes = [make_scene(scene_name, frame=200 + i) for i in range(n_frames)]
    s0 = scenes[0]
    out = {"scene": scene_name, "frames": n_frames}
    chains = {"cd_s10_d8": {}, "cd_s30_d16": dict(dirs=16, steps=30), "st_s10_d8": dict(support=2, st_t=0.1),
              "fixed_9x9": dict(support=0, r_affine=4), "fixed_13x13": dict(support=0, r_affine=6),
              "fixed_15x15": dict(support=0, r_affine=7), "learned": dict(learned=1)}
    for name, params in chains.items():
        pipe = Pipeline(s0.camera, s0.W, s0.H, **params)
        try:
            bufs = []
            for s in scenes:
                b = pipe.buffers()
                pipe.run_frame(pipe.upload(s.disp), b)
                bufs.append(b)
            torch.cuda.synchronize()
            sn.sn_check_device(pipe.ctx)
            out[name] = gt_error_deg(bufs, scenes)
        finally:
            pipe.close()
    ctx = sn.sn_create(s0.camera, s0.W, s0.H, sn.default_params())
    try:
        for name in ("pca_9x9", "cross"):
            bufs = []
            for s in scenes:
                d = sn.empty_image(s0.H, s0.W, torch.float32)
                d.copy_(torch.from_numpy(s.disp))

                class _O:
                    pass
                o = _O()
                o.normals, o.mask = sn.empty_planes(3, s0.H, s0.W), sn.empty_image(s0.H, s0.W, torch.uint8)
                if name == "cross":
                    sn.sn_cross_normals(ctx, d, o.normals, o.mask)
                else:
                    sn.sn_pca_normals(ctx, d, 4, o.normals, o.mask)
                bufs.append(o)
            torch.cuda.synchronize()
            out[name] = gt_error_deg(bufs, scenes)
        sn.sn_check_device(ctx)
    finally:
        sn.sn_destroy(ctx)
    return out


MIXED_SIZES = ("planes_320x240", "planes_640x480", "mixed_1482x994", "driving_2048x1024")


def run_mixed_batch(args, seed=0):
    """64 frames, 16 of each size (4 distinct seeded scenes per size, each
    used 4 times) in seeded shuffled order: the plain and the learned chain,
    each whole batch captured as one CUDA graph (one launch per step, the
    frames spread over the graph's streams).  MPix/s over the 63,268,160
    pixels of a step and the mean angular error against ground truth."""
    import torch
    from scenes import make_scene
    from paper_2504_15121_gb300 import Pipeline
    rng = np.random.default_rng([4, seed])
    scenes = {n: [make_scene(n, frame=100 + i) for i in range(4)] for n in MIXED_SIZES}
    order = [(n, i % 4) for n in MIXED_SIZES for i in range(16)]
    order = [order[k] for k in rng.permutation(len(order))]
    px = sum(scenes[n][0].W * scenes[n][0].H for n, _ in order)
    out = {"frames": len(order), "pixels_per_step": int(px),
           "order": "seeded shuffle of 16 frames of each of " + ", ".join(MIXED_SIZES)}
    for form, params in (("plain_f32", {}), ("learned_f32", dict(learned=1))):
        pipes = {n: Pipeline(scenes[n][0].camera, scenes[n][0].W, scenes[n][0].H, **params) for n in MIXED_SIZES}
        try:
            disp = {n: [pipes[n].upload(sc.disp) for sc in scenes[n]] for n in MIXED_SIZES}
            bufs = [pipes[n].buffers() for n, _ in order]
            main = torch.cuda.current_stream()
            streams = [torch.cuda.Stream() for _ in range(args.streams)]

            def step():
                cur = torch.cuda.current_stream()
                ev = cur.record_event()
                for st in streams:
                    st.wait_event(ev)
                for k, (n, i) in enumerate(order):
                    pipes[n].run_frame(disp[n][i], bufs[k], stream=streams[k % len(streams)], write_den=False)
                for st in streams:
                    cur.wait_stream(st)
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream()
            with torch.cuda.stream(cap):
                graph.capture_begin()
                step()
                graph.capture_end()
            torch.cuda.synchronize()
            for _ in range(2):
                graph.replay()
            torch.cuda.synchronize()
            steps = max(3, args.steps // 4)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(main)
            for _ in range(steps):
                graph.replay()
            t1.record(main)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            errs = []
            for k, (n, i) in enumerate(order):
                e = gt_error_deg([bufs[k]], [scenes[n][i]])
                errs.append((e["mean"], e["pixels"], e["certified"]))
            npx = sum(p for _, p, _ in errs)
            out[form] = {"value": steps * px / (ms / 1e3) / 1e6, "unit": "MPix/s", "ms_per_step": ms / steps,
                         "graph_launches_per_step": 1,
                         "gt_error_deg": sum(m * p for m, p, _ in errs) / max(npx, 1),
                         "certified": float(np.mean([c for _, _, c in errs]))}
            del graph
        finally:
            for pp in pipes.values():
                pp.close()
    out["learned_vs_plain"] = out["learned_f32"]["value"] / out["plain_f32"]["value"]
    return out


# compulsory bytes per pixel of each stage entry point (FP32 form)
STAGE_BYTES = {"sn_denoise": 4 + 4 + 1, "sn_affine_normals": 4 + 4 + 12 + 1, "sn_components": 4 + 4,
               "sn_pointcloud": 4 + 1 + 12}


def time_stage_calls(scenes, args):
    """Each stage entry point on its own (default method, same scenes, one
    stream): device time per frame from CUDA events around a run of calls,
    MPix/s and the fraction of the measured HBM bandwidth its compulsory
    bytes reach."""
    import torch
    from paper_2504_15121_gb300 import sn
    peaks, _ = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    s0 = scenes[0]
    W, H = s0.W, s0.H
    ctx = sn.sn_create(s0.camera, W, H, sn.default_params())
    out = {}
    try:
        disp = []
        for s in scenes:
            t = sn.empty_image(H, W, torch.float32)
            t.copy_(torch.from_numpy(s.disp))
            disp.append(t)
        den = [sn.empty_image(H, W, torch.float32) for _ in scenes]
        m1 = [sn.empty_image(H, W, torch.uint8) for _ in scenes]
        nrm = sn.empty_planes(3, H, W)
        m2 = sn.empty_image(H, W, torch.uint8)
        lab = sn.empty_image(H, W, torch.int32)
        pts = sn.empty_planes(3, H, W)
        for i in range(len(scenes)):
            sn.sn_denoise(ctx, disp[i], den[i], m1[i])
        calls = {
            "sn_denoise": lambda i: sn.sn_denoise(ctx, disp[i], den[i], m1[i]),
            "sn_affine_normals": lambda i: sn.sn_affine_normals(ctx, disp[i], den[i], nrm, m2),
            "sn_components": lambda i: sn.sn_components(ctx, disp[i], lab, None),
            "sn_pointcloud": lambda i: sn.sn_pointcloud(ctx, den[i], m1[i], pts),
        }
        reps = max(8, args.steps // 8)
        for name, call in calls.items():
            for i in range(4):
                call(i % len(scenes))
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for i in range(reps):
                call(i % len(scenes))
            t1.record()
            torch.cuda.synchronize()
            us = t0.elapsed_time(t1) / reps * 1e3
            gbs = STAGE_BYTES[name] * W * H / (us * 1e-6) / 1e9
            out[name] = {"us_per_frame": us, "mpix_s": W * H / us, "algo_bytes_per_px": STAGE_BYTES[name],
                         "hbm_frac": gbs / hbm}
        sn.sn_check_device(ctx)
    finally:
        sn.sn_destroy(ctx)
    return out


def gt_error_deg(outs, scenes):
    """Mean angular error (degrees) of the normals against the generator's
    ground truth, over the foreground pixels with a valid normal of the first
    frame of each distinct scene (read back after the timed region), and the
    fraction of valid pixels the learned gate certified."""
    import torch
    errs, cert, near = [], [], []
    for s, out in zip(scenes, outs):
        m = out.mask.cpu().numpy()
        if out.normals.dtype == torch.int16:
            n = out.normals.cpu().numpy()[..., :3].astype(np.float64) / 32767.0
        else:
            n = np.moveaxis(out.normals.cpu().numpy().astype(np.float64), 0, -1)
        ok = ((m & 2) > 0) & ~s.background
        a, b = n[ok], s.gt_normal[ok].astype(np.float64)
        ang = np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1)))
        errs.append(ang)
        near.append(near_edge(s.prim, EDGE_BAND)[ok])
        cert.append(((m & 8) > 0).sum() / max(((m & 1) > 0).sum(), 1))
    e, ne = np.concatenate(errs), np.concatenate(near)
    return {"mean": float(e.mean()), "median": float(np.median(e)), "pixels": int(e.size),
            f"mean_within_{EDGE_BAND}px_of_a_surface_edge": float(e[ne].mean()) if ne.any() else None,
            "mean_elsewhere": float(e[~ne].mean()) if (~ne).any() else None,
            "edge_band_pixels": int(ne.sum()),
            "certified": float(np.mean(cert)), "scenes": len(errs)}


def near_edge(prim, r):
    """Pixels within r (Chebyshev distance) of a change of the generator's
    primitive id (a surface edge, including the edge to the background)."""
    e = np.zeros(prim.shape, bool)
    e[:, 1:] |= prim[:, 1:] != prim[:, :-1]
    e[:, :-1] |= prim[:, 1:] != prim[:, :-1]
    e[1:, :] |= prim[1:, :] != prim[:-1, :]
    e[:-1, :] |= prim[1:, :] != prim[:-1, :]
    for axis in (0, 1):  # dilation by a (2r + 1)-wide box, one axis at a time
        d = e.copy()
        for k in range(1, r + 1):
            d[tuple(slice(k, None) if a == axis else slice(None) for a in range(2))] |= \
                e[tuple(slice(None, -k) if a == axis else slice(None) for a in range(2))]
            d[tuple(slice(None, -k) if a == axis else slice(None) for a in range(2))] |= \
                e[tuple(slice(k, None) if a == axis else slice(None) for a in range(2))]
        e = d
    return e


SERVING_CAMERAS = [("planes_640x480", 120.0)] * 2 + [("mixed_1482x994", 30.0)] * 4 + \
    [("driving_2048x1024", 30.0)] * 2


def run_serving(args):
    """The serving workload: 8 simulated cameras (2x 640x480 at 120 Hz,
    4x 1482x994 at 30 Hz, 2x 2048x1024 at 30 Hz), Poisson arrivals, one
    CUDA graph per request slot, 4 streams; latency from arrival to result
    ready on the device.  Offered rate x1 for --serve-seconds, then a rate
    sweep; plain FP32 chain, FP16 in / snorm16 out chain, and the learned
    chain with FP16 in / snorm16 out."""
    import numpy as np
    import torch
    from paper_2504_15121_gb300 import serve, sn
    from scenes import make_scene
    pools_src = {}
    for name, _ in SERVING_CAMERAS:
        if name not in pools_src:
            pools_src[name] = [make_scene(name, frame=100 + k) for k in range(2)]
    out = {}
    for form, params, pick in (
            ("plain_f32", {}, lambda s: s.disp),
            ("f16_snorm16", dict(in_dtype=sn.SN_IN_F16, normal_fmt=sn.SN_NORMALS_SNORM16X4),
             lambda s: s.disp.astype(np.float16)),
            # the learned + FP16 chain of the serving workload
            ("learned_f16_snorm16", dict(learned=1, in_dtype=sn.SN_IN_F16, normal_fmt=sn.SN_NORMALS_SNORM16X4),
             lambda s: s.disp.astype(np.float16))):
        cams, pools = [], []
        for name, rate in SERVING_CAMERAS:
            ss = pools_src[name]
            cams.append(serve.camera(ss[0].W, ss[0].H, ss[0].camera, rate_hz=rate, **params))
            pools.append([torch.from_numpy(np.ascontiguousarray(pick(s))).pin_memory() for s in ss])
        srv = serve.Server(cams, memory_budget=6 << 30, max_slots_per_camera=6, n_streams=4, queue_depth=256)
        try:
            res = {"x1": srv.simulate(pools, duration_s=args.serve_seconds, rate_scale=1.0, seed=1)}
            # rate sweep: x48 offers more than the device sustains (saturation)
            for k in (8, 24, 48):
                res[f"x{k}"] = srv.simulate(pools, duration_s=1.0, rate_scale=float(k), seed=k)
            srv.check()
        finally:
            srv.close()
        out[form] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                     for k, v in res.items()}
    out["how"] = ("8 cameras: 2x 640x480 @120 Hz, 4x 1482x994 @30 Hz, 2x 2048x1024 @30 Hz; Poisson "
                  "arrivals; latency = arrival (pinned host frame) -> outputs ready on device; "
                  "x8/x24/x48 = every camera's rate multiplied (x48 saturates)")
    return out


# sources each kernel's build depends on (the traffic figure is void once
# any of them has changed since the capture)
KERNEL_SOURCES = {"frame": ("sn_frame.cu", "sn_pixel.cuh", "sn_device.cuh", "sn_umma.cuh", "sn_internal.h")}


def kernel_source_sha(kernel: str):
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2504_15121_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch (read + write, write-back included) from the
    committed ncu summary profiles/traffic.json, if it was taken on the
    current sources of this kernel; None otherwise."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f).get(kernel)
        if not t or t.get("source_sha") != kernel_source_sha(kernel):
            return None
        return t
    except Exception:
        return None


def host_link_gbs(nbytes=64 << 20, reps=10):
    """Copy rate between pinned host memory and the device, each direction
    alone (CUDA events around `reps` copies of `nbytes`)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    for name, dst, src in (("d2h_gbs", h, d), ("h2d_gbs", d, h)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        out[name] = nbytes * reps / (a.elapsed_time(b) / 1e3) / 1e9
    return out


def run_e2e(pipe, scenes, args, world, dist):
    import torch
    from paper_2504_15121_gb300 import sn
    W, H = pipe.W, pipe.H
    F = args.frames
    host_in = []
    for s in scenes:
        t = torch.from_numpy(s.disp).pin_memory()
        host_in.append(t)
    NS = 2  # the host copies are bandwidth-bound: 2 streams measured best (2: 5.9, 4: 5.6, 8: 5.4 GPix/s)
    host_out = [pipe.host_buffers() for _ in range(NS)]
    streams = [torch.cuda.Stream() for _ in range(NS)]
    h2d = W * H * 4
    d2h = W * H * (12 + 12 + 4 + 1) + 4

    def frame(f):
        # the C ABI on host buffers: copy in, sn_run_frame, copy out, all on
        # the stream (the context's staging buffers rotate)
        i = f % NS
        pipe.run_frame_host(host_in[f % len(host_in)], host_out[i], stream=streams[i])

    steps = max(3, args.steps // 4)
    for f in range(NS * F):
        frame(f)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        for f in range(F):
            frame(f)
        torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, dist)
    link = host_link_gbs()
    # the host link bounds the end-to-end rate: per frame, h2d bytes one way
    # and d2h bytes the other, each at its measured copy rate
    bound = W * H / max(h2d / (link["h2d_gbs"] * 1e9), d2h / (link["d2h_gbs"] * 1e9)) / 1e6
    value = whole_job_mpix(world, steps * F * W * H, dt * 1e3)
    return {"value": value, "unit": "MPix/s", "h2d_bytes_per_step": F * h2d,
            "d2h_bytes_per_step": F * d2h, "steps": steps,
            "link": dict(link, bound_mpix_s=bound * world, frac=value / (bound * world)),
            "how": "sn_run_frame_host (C ABI on host buffers): pinned host disparity -> device, "
                   "the chain, normals/points/labels/mask/count -> pinned host; "
                   f"{NS} streams taking frames in turn; host wall clock with a device sync per step"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
