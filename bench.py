#!/usr/bin/env python3
"""Benchmark of the detect pipeline (Gsites/s) on GB300.

Default workload: 64 frames of a 1024x1024 periodic smoothed-noise lattice
(sigma 4, threshold 0.5, shear 0.005 per frame + N(0, 0.01)), processed in
order through a frame-sequence batch (every stage launched once for all 64
frames, 67.1M sites per push). One timed step = R consecutive pushes of the
sequence, R chosen from the warm-up so that the K timed steps last at least
a second (stated in the line); the plain one-frame-per-call path is timed too
and reported beside it. The 256 MiB of input frames is resident in HBM and
larger than L2 (129 MB), so every frame is read cold.

The same line also carries the batched form (256 uneven lattices, one push
per frame, against the same lattices one by one) and the served form (64
simulations, seeded Poisson arrivals, against the plain per-frame FIFO on the
same trace, latency from arrival), with a served rate sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Multi-GPU (torchrun): every rank runs an independent
replica on its own GPU (weak scaling, no collective on the data path); the
time is the max over ranks. ``--impl reference`` times the CPU oracle as it
stands on the host cores (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1607_00908_gb300 import inputs  # noqa: E402

METRIC = "Gsites/s full detect pipeline"
UNIT = "Gsites/s"

# The pipeline's per-site traffic floor: the field is read once (4) and the
# Voronoi owners, the one per-site result kept in HBM, are written once (4);
# labels are kept per run, not per site.
PIPELINE_BYTES_PER_SITE = 8.0
# The metric's own % HBM figure counts 16 B/site (field read, previous-label
# read, label write, owner write: the per-site traffic of a pipeline that
# stores per-site labels), whatever this implementation actually moves.
METRIC_BYTES_PER_SITE = 16.0

# Measured DRAM bytes (read + write) per site of a stage's kernels, from one
# ncu capture of the current kernels on 48 frames of this workload
# (profiles/site_kernels_c1.txt); scaled to the bench launch for
# roofline.traffic. The owner stage's entry depends on its patch layout
# (VD_PATCH_*); a stage or layout not captured, or whose kernels changed since
# the capture, reports null.
TRAFFIC_BYTES_PER_SITE = {0: 4.193, 2: 0.278, 3: {0: 2.869}, 4: 4.342}

# Issue-slot use (smsp__issue_active, % of peak) of the same kernels in the
# same capture: the kernels are bound by instruction issue or latency, not by
# DRAM, and this says how close to the issue limit they run.
ISSUE_ACTIVE_PCT = {0: 64.7, 2: 49.5, 3: {0: 73.1}, 4: 57.9}


def per_stage(table, stage, patch):
    v = table.get(stage)
    return v.get(patch) if isinstance(v, dict) else v


def workload(name: str, n_frames: int | None):
    if name == "c1":
        n = n_frames or 64
        return f"1024x1024 smoothed noise sigma 4, {n} frames (shear 0.005 + N(0,0.01))", list(inputs.workload_c1(1, n))
    if name == "c0":
        return "128x128 smoothed noise sigma 3, 2 frames", inputs.workload_c0(1)
    if name == "c2":
        n = n_frames or 16
        return f"4096x4096 RSA droplets r~U[8,12], {n} frames (shear 1e-3 + N(0,0.3))", \
            [F for F, _ in inputs.workload_c2(1, n)]
    raise SystemExit(f"unknown workload {name}")


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        load = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_ranks(world: int, local: int, backend: str | None = None) -> None:
    """One process per GPU under torchrun: replicas that exchange only timings
    and unit counts (NCCL on GPUs, gloo on the host)."""
    if world <= 1:
        return
    import torch
    import torch.distributed as dist
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    if not dist.is_initialized():
        dist.init_process_group(backend)


def _reduce_over_ranks(x: float, world: int, op_name: str) -> float:
    """All-reduce of one host number over the ranks (replicas only exchange
    their timings and unit counts, never data of the path). The tensor lives
    where the process group's backend wants it: CUDA for NCCL, host for gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return _reduce_over_ranks(x, world, "MAX")


def sum_over_ranks(x: float, world: int) -> float:
    return _reduce_over_ranks(x, world, "SUM")


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(frames, budget_s: float = 15.0, min_frames: int = 2):
    """The CPU oracle as it stands, single-threaded, on a bounded sample of the workload."""
    import oracle
    Ly, Lx = frames[0].shape
    det = oracle.Detector(Lx, Ly, workers=1)
    t0 = time.perf_counter()
    n = 0
    for F in frames:
        det.push(F)
        n += 1
        if n >= min_frames and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n * Lx * Ly / dt / 1e9, n, dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    desc, frames = workload(args.workload, args.frames)
    import oracle
    Ly, Lx = frames[0].shape
    det = oracle.Detector(Lx, Ly, workers=1)
    # a step is one frame of the workload through the whole oracle pipeline
    k = 0
    for _ in range(args.warmup):
        det.push(frames[k % len(frames)])
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        det.push(frames[k % len(frames)])
        k += 1
    dt = time.perf_counter() - t0
    value = args.steps * Lx * Ly / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc + " (one frame per step)", "l2_policy": "host CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} frames of the workload after {args.warmup} warm-up frames"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def stage_bytes(sequence: bool):
    """Algorithmic bytes per site of the stages that touch every site.

    stage 0 threshold pass + tile union-find: field read 4, foreground
            bit write 1/8 (the union-find re-reads the bits, from L2)
    stage 2 run labels + overlaps: foreground bits of the frame and of its
            past frame, 1/8 + 1/8 (run tables are per run, not per site)
    stage 3 Voronoi owners: owner write 4
    stage 4 links: owner read 4
    """
    return {0: 4.125, 2: 0.25, 3: 4.0, 4: 4.0}


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def roofline_of(stage_ms, names, launches_per_stage, sites_per_launch, sequence, peak, peak_kind, patch=0):
    sb = stage_bytes(sequence)
    dom = max(sb, key=lambda k: stage_ms[k])
    avg_ms = stage_ms[dom] / launches_per_stage
    bytes_per_launch = sb[dom] * sites_per_launch
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    traffic = per_stage(TRAFFIC_BYTES_PER_SITE, dom, patch)
    return {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": traffic * sites_per_launch if traffic is not None else None,
            "issue_active_pct_ncu": per_stage(ISSUE_ACTIVE_PCT, dom, patch),
            "bytes_per_site": sb[dom], "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
            "stage_ms_per_launch": {names[k]: stage_ms[k] / launches_per_stage for k in range(len(names))}}


def plain_frames_c2(world, s, e0, e1, n_frames=4, reps=3):
    """The plain per-frame path on 4096^2 droplet frames: vd_push_frame, one
    frame per call (graph replay), ms per frame over reps passes."""
    import torch
    from paper_1607_00908_gb300 import vd
    frames = [F for F, _ in inputs.workload_c2(1, n_frames)]
    Ly, Lx = frames[0].shape
    dev = [torch.from_numpy(F).cuda() for F in frames]
    det = vd.Detector(Lx, Ly, stream=s.cuda_stream)
    for F in dev:
        det.push(F)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        for F in dev:
            det.push(F)
    e1.record(s)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    det.close()
    return {"value": world * Lx * Ly * n_frames * reps / (ms / 1e3) / 1e9, "unit": UNIT,
            "ms_per_frame": ms / reps / n_frames, "frames": n_frames * reps,
            "workload": f"{Lx}x{Ly} RSA droplets r~U[8,12], {n_frames} frames, each pushed {reps} times",
            "path": "vd_push_frame per frame (graph replay)"}


def pick_tuning(args, b, dev, s):
    """The autotuner's choice for batch b, or the setting given as
    --tuning PATCH,BUCKET_PCT,RING0 (e.g. 8x8,100,9)."""
    from paper_1607_00908_gb300 import autotune, vd
    if args.tuning == "auto":
        return autotune.tune(b, dev, s, use_cache=False)
    patch, bucket, ring = args.tuning.split(",")
    t = dict(voronoi_patch=getattr(vd, "VD_PATCH_" + patch), bucket_pct=int(bucket), ring0=int(ring))
    b.set_tuning(**t)
    return dict(t, fixed=True)


def run_ours(args, world, rank, local):
    c3 = None if args.no_c3 else c3_host_frames(rank)   # host cores, before the first GPU call
    import torch
    from paper_1607_00908_gb300 import vd

    torch.cuda.set_device(local if world > 1 else 0)
    vd.lib()
    desc, frames = workload(args.workload, args.frames)
    n = len(frames)
    Ly, Lx = frames[0].shape
    sites_per_step = n * Lx * Ly
    s = torch.cuda.Stream()
    dev = [torch.from_numpy(F).cuda() for F in frames]
    torch.cuda.synchronize()
    peak, peak_kind = read_peaks()

    # ---- headline: the whole frame sequence per push (one launch per stage);
    # a timed step is R pushes, R set from the warm-up so that the K steps
    # last at least args.min_seconds ----
    seq = vd.Batch([(Lx, Ly)], sequence=n, stream=s.cuda_stream)
    tuned = pick_tuning(args, seq, dev, s)   # launch shapes for this workload (untimed)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.warmup):
        seq.push(dev)
    e1.record(s)
    torch.cuda.synchronize()
    push_ms = max(e0.elapsed_time(e1) / max(1, args.warmup), 1e-3)
    reps = max(1, int(np.ceil(args.min_seconds * 1e3 / (args.steps * push_ms))))
    reps = int(max_over_ranks(float(reps), world))
    sites_per_push = sites_per_step
    sites_per_step = reps * sites_per_push
    clocks = Clocks(local)
    clocks.start()
    launches0 = seq.timing()[2]
    barrier(world)
    torch.cuda.synchronize()
    nvtx_push("vd_timed")   # lets a profiler select the timed pushes
    e0.record(s)
    for _ in range(args.steps * reps):
        seq.push(dev)
    e1.record(s)
    torch.cuda.synchronize()
    nvtx_pop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = seq.timing()[2] - launches0
    ms_max = max_over_ranks(ms, world)
    value = world * sites_per_step * args.steps / (ms_max / 1e3) / 1e9

    # ---- roofline: per-stage CUDA events on the library stream, same work ----
    seq.set_timing(True)
    seq.timing()
    n_timed = max(args.steps, 20)
    for _ in range(n_timed):
        seq.push(dev)
    stage_ms, names, _, _ = seq.timing()
    seq.set_timing(False)
    roofline = roofline_of(stage_ms, names, n_timed, sites_per_push, n > 1, peak, peak_kind,
                           seq.tuning()["voronoi_patch"])
    roofline["pipeline_frac_8B_per_site"] = value * PIPELINE_BYTES_PER_SITE / peak
    roofline["pct_hbm_16B_per_site"] = 100.0 * value * METRIC_BYTES_PER_SITE / peak

    # ---- end to end through the C ABI with host buffers: every step's frames
    # are copied from pinned host memory (staged on the batch's copy stream
    # while the previous step runs) and every frame's results are read back ----
    host = torch.from_numpy(np.stack(frames)).pin_memory()   # the sequence's frames, one pinned array
    ptrs = [host[i].data_ptr() for i in range(n)]
    e2e_steps = max(2, args.steps)
    d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq.stage_host_ptrs(ptrs)
    seq.push_staged()
    for k in range(e2e_steps):
        if k + 1 < e2e_steps:
            seq.stage_host_ptrs(ptrs)
        allc = seq.changes_all()
        d2h += 20 * n + 16 * len(allc["breaking"]) + 8 * len(allc["arising"]) + len(allc["active"])
        if k + 1 < e2e_steps:
            seq.push_staged()
    torch.cuda.synchronize()
    e2e_dt = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * sites_per_push * e2e_steps / e2e_dt / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 4 * sites_per_push, "d2h_bytes_per_step": int(d2h / e2e_steps),
           "step": f"one push of the {n}-frame sequence (host frames in, every frame's results out)",
           "path": "vd_batch_stage_host (double-buffered, copy stream) + vd_batch_push_staged + "
                   "vd_batch_get_changes_all for every step"}
    seq.close()

    # ---- options beyond the default steps a1-a8, on the same workload: the
    # event classes of Section 3.2.4, the centre match of Section 3.2.3 (with
    # events), the paper's vertex link rule of Section 3.2.2, 8-connectivity ----
    variants = {}
    for name, opts in (("events", dict(events=True)),
                       ("centroid_match_r8_events", dict(events=True, match_rule=vd.VD_MATCH_CENTROID,
                                                         match_radius=8)),
                       ("vertex_links", dict(edge_rule=vd.VD_EDGE_VERTEX)),
                       ("connectivity_8", dict(connectivity=8))):
        vb = vd.Batch([(Lx, Ly)], sequence=n, stream=s.cuda_stream, **opts)
        for _ in range(max(1, args.warmup)):
            vb.push(dev)
        torch.cuda.synchronize()
        vsteps = max(1, min(args.steps, 5))
        e0.record(s)
        for _ in range(vsteps):
            vb.push(dev)
        e1.record(s)
        torch.cuda.synchronize()
        vms = max_over_ranks(e0.elapsed_time(e1), world)
        # per-stage CUDA events on the library stream, separate untimed pushes
        vb.set_timing(True)
        vb.timing()
        for _ in range(vsteps):
            vb.push(dev)
        vst, vnames, _, _ = vb.timing()
        vb.set_timing(False)
        variants[name] = {"value": world * sites_per_push * vsteps / (vms / 1e3) / 1e9, "unit": UNIT,
                          "ms_per_step": vms / vsteps, "steps": vsteps,
                          "stage_ms_per_step": {vnames[k]: vst[k] / vsteps for k in range(len(vnames))}}
        vb.close()

    # ---- the plain per-frame path (vd_push_frame, one frame per call) ----
    det = vd.Detector(Lx, Ly, stream=s.cuda_stream)
    for F in dev[: min(n, 4)]:
        det.push(F)
    torch.cuda.synchronize()
    plain_steps = max(1, min(args.steps, 3))
    e0.record(s)
    for _ in range(plain_steps):
        for F in dev:
            det.push(F)
    e1.record(s)
    torch.cuda.synchronize()
    plain_ms = max_over_ranks(e0.elapsed_time(e1), world)
    plain = {"value": world * sites_per_push * plain_steps / (plain_ms / 1e3) / 1e9, "unit": UNIT,
             "path": "vd_push_frame per frame (graph replay)", "ms_per_frame": plain_ms / plain_steps / n}
    det.close()
    del dev
    torch.cuda.synchronize()
    plain_c2 = None if args.no_c2_plain else plain_frames_c2(world, s, e0, e1)

    # ---- the batched and served forms (the metric's "batched/served vs plain") ----
    batched = measure_batched(world, *c3) if c3 is not None else None
    c3 = None
    served = None if args.no_c4 else measure_served(world, rank, args.serve_rate, args.serve_seconds)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, nfr, dt = cpu_baseline(frames)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"first {nfr} frames of the workload, {dt:.1f} s single-threaded"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": desc, "sites_per_step": sites_per_step, "pushes_per_step": reps,
                       "path": f"vd_batch_create_sequence: {n} frames per push, one launch per stage; "
                               f"a step is {reps} consecutive pushes of the sequence",
                       "tuning": tuned,
                       "l2_policy": "inputs larger than L2 (each step reads all frames once)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "plain_per_frame": plain, "plain_per_frame_c2": plain_c2, "options": variants,
        }
        if batched is not None:
            line["batched_c3"] = batched
        if served is not None:
            line["served_c4"] = served
        print(json.dumps(line), flush=True)


def measure_served(world, rank, rate: float, seconds: float, sweep=(1.5, 2.0, 3.0, 4.0, 6.0, 8.0),
                   plain_sweep=(1.5, 2.0), sweep_seconds: float = 2.0):
    """Served form: 64 simulations, seeded Poisson arrivals, 40 GB budget. The
    same trace runs through the server (continuous batching) and through the
    plain per-frame path (vd_push_frame FIFO, one stream); latency is counted
    from each frame's arrival. Shorter traces at multiples of the rate give
    each arm's throughput against p99; the comparison at equal p99 takes, for
    a p99 bound, the best throughput each arm reached within it."""
    import torch
    from paper_1607_00908_gb300 import inputs, serve

    params = inputs.serve_sims(64, 5 + rank)
    sims = [(L, rec) for L, rec, _ in params]
    host_pools = serve.make_pools([L for L, _ in sims], 4)
    dev_pools = {k: [torch.from_numpy(F).cuda() for F in v] for k, v in host_pools.items()}
    del host_pools
    budget = int(40e9)
    trace = serve.poisson_trace(64, rate, seconds, 5 + rank)
    served = serve.run(sims, dev_pools, trace, max_batch=64, budget_bytes=budget)
    plain = serve.run_plain(sims, dev_pools, trace)
    offered = sum(sims[s_][0] ** 2 for _, s_ in trace) / seconds / 1e9

    def point(r, rt, sec):
        return {"rate": rt, "seconds": sec, "gsites_per_s": r["gsites_per_s"], "p50_ms": r["p50_ms"],
                "p99_ms": r["p99_ms"]}

    s_pts, p_pts = [point(served, rate, seconds)], [point(plain, rate, seconds)]
    for m in sweep:
        tr = serve.poisson_trace(64, rate * m, sweep_seconds, 100 + rank + int(10 * m))
        s_pts.append(point(serve.run(sims, dev_pools, tr, max_batch=64, budget_bytes=budget), rate * m,
                           sweep_seconds))
    for m in plain_sweep:
        tr = serve.poisson_trace(64, rate * m, sweep_seconds, 100 + rank + int(10 * m))
        p_pts.append(point(serve.run_plain(sims, dev_pools, tr), rate * m, sweep_seconds))
    tot = lambda v: sum_over_ranks(v, world)

    def best_within(pts, bound):
        ok = [p_ for p_ in pts if p_["p99_ms"] <= bound]
        return max((p_["gsites_per_s"] for p_ in ok), default=0.0)

    equal_p99 = []
    for bound in (plain["p99_ms"], 5.0):
        equal_p99.append({"p99_bound_ms": bound, "served_gsites_per_s": tot(best_within(s_pts, bound)),
                          "plain_gsites_per_s": tot(best_within(p_pts, bound))})
    return {
        "workload": "64 simulations, L in {512,1024,2048,4096}, noise/RSA recipes alternating, "
                    f"Poisson arrivals {rate:.0f} frames/s for {seconds} s, 40 GB budget",
        "offered_gsites_per_s": tot(offered), "arrivals": len(trace),
        "served": {**served, "gsites_per_s": tot(served["gsites_per_s"])},
        "plain_fifo": {**plain, "gsites_per_s": tot(plain["gsites_per_s"]),
                       "path": "vd_push_frame per frame, one context per simulation, one stream, arrival order"},
        "latency_from": "arrival (trace time on the library clock)",
        "rate_sweep": {"served": s_pts, "plain_fifo": p_pts},
        "at_equal_p99": equal_p99,
    }


def run_served(args, world, rank, local):
    import torch
    from paper_1607_00908_gb300 import vd

    torch.cuda.set_device(local if world > 1 else 0)
    vd.lib()
    r = measure_served(world, rank, args.serve_rate, args.serve_seconds)
    if rank == 0:
        s_ = r["served"]
        line = {
            "metric": METRIC + " (served)", "value": s_["gsites_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": s_["steps"], "warmup": 0, "ms_per_step": 1e3 * s_["wall_s"] / max(1, s_["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": r["workload"]}, **r,
        }
        print(json.dumps(line), flush=True)


def _c3_frames(spec):
    from paper_1607_00908_gb300 import inputs
    L, sigma, seed = spec
    return list(inputs.noise_frames(L, sigma, 8, 0.02, seed))


def c3_host_frames(rank: int):
    """The batched workload's frames, generated on the host cores (spawned pool)."""
    import multiprocessing as mp

    from paper_1607_00908_gb300 import inputs

    specs = inputs.batch_instances(256, seed=3 + rank)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        host = pool.map(_c3_frames, specs)
    return specs, host


def measure_batched(world, specs, host):
    """Batched form: 256 lattices of uneven size advanced together, one
    vd_batch_push per frame (8 frames), against the same lattices one by one
    through vd_push_frame."""
    import torch
    from paper_1607_00908_gb300 import vd

    from paper_1607_00908_gb300 import autotune

    n, nf = len(specs), 8
    dev = [[torch.from_numpy(F).cuda() for F in fr] for fr in host]
    sites_per_step = sum(L * L for L, _, _ in specs)
    s = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(b):
        for f in range(nf):   # warm-up pass over the 8 frames
            b.push([dev[i][f] for i in range(n)])
        torch.cuda.synchronize()
        barrier(world)
        e0.record(s)
        for f in range(nf):
            b.push([dev[i][f] for i in range(n)])
        e1.record(s)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world)

    # the default launch shapes, then the shapes the autotuner picks on frame 0
    b = vd.Batch([(L, L) for L, _, _ in specs], stream=s.cuda_stream)
    ms_default = timed(b)
    b.close()
    b = vd.Batch([(L, L) for L, _, _ in specs], stream=s.cuda_stream)
    tuned = autotune.tune(b, [dev[i][0] for i in range(n)], s, use_cache=False)
    ms = timed(b)
    b.close()
    dets = [vd.Detector(L, L, stream=s.cuda_stream) for L, _, _ in specs]
    for i in range(n):
        for f in range(nf):
            dets[i].push(dev[i][f])
    torch.cuda.synchronize()
    e0.record(s)
    for i in range(n):
        for f in range(nf):
            dets[i].push(dev[i][f])
    e1.record(s)
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(e0.elapsed_time(e1), world)
    for d in dets:
        d.close()
    del dev
    total_sites = sum_over_ranks(float(sites_per_step), world)
    value = total_sites * nf / (ms / 1e3) / 1e9
    plain = total_sites * nf / (ms_plain / 1e3) / 1e9
    return {"value": value, "unit": UNIT, "ms_per_frame_step": ms / nf, "sites_per_frame_step": sites_per_step,
            "tuning": tuned, "default_shapes": {"value": total_sites * nf / (ms_default / 1e3) / 1e9, "unit": UNIT,
                                                "ms_per_frame_step": ms_default / nf},
            "workload": "256 lattices, L in {256,384,512,768,1024,1536,2048}, smoothed noise sigma U[2,6], "
                        "8 frames, one vd_batch_push per frame",
            "plain": {"value": plain, "unit": UNIT, "ms_per_frame_step": ms_plain / nf,
                      "path": "vd_push_frame per lattice and frame, instance after instance"},
            "speedup_vs_plain": value / plain}


def run_batched_c3(args, world, rank, local):
    specs, host = c3_host_frames(rank)   # before the first GPU call
    import torch
    from paper_1607_00908_gb300 import vd

    torch.cuda.set_device(local if world > 1 else 0)
    vd.lib()
    r = measure_batched(world, specs, host)
    if rank == 0:
        line = {
            "metric": METRIC + " (batched)", "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": 8,
            "warmup": 8, "ms_per_step": r["ms_per_frame_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": r["workload"], "sites_per_step": r["sites_per_frame_step"],
                       "parallelism": f"replicas x{world}"},
            "plain": r["plain"], "speedup_vs_plain": r["speedup_vs_plain"],
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="served workload: arrivals per second")
    ap.add_argument("--min-seconds", type=float, default=1.5,
                    help="headline: the K timed steps last at least this long (pushes per step set from the warm-up)")
    ap.add_argument("--tuning", default="auto",
                    help="headline launch shapes: auto (the autotuner) or PATCH,BUCKET_PCT,RING0, e.g. 8x8,100,9")
    ap.add_argument("--no-c2-plain", action="store_true", help="leave the per-frame 4096^2 figure out of the line")
    ap.add_argument("--no-c3", action="store_true", help="leave the batched form out of the default line")
    ap.add_argument("--no-c4", action="store_true", help="leave the served form out of the default line")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)   # rank 0 alone; the others exit without work
        return
    init_ranks(world, local)
    if args.workload == "c4":
        run_served(args, world, rank, local)
    elif args.workload == "c3":
        run_batched_c3(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
