"""Served-form workload: frames of many simulations arriving as a Poisson stream.

64 simulations with L in {512, 1024, 2048, 4096} (seeded), alternating the
smoothed-noise recipe (sigma 4) and the RSA droplet recipe; frames arrive as
one seeded Poisson process of aggregate rate `rate` frames/s, each arrival
picking a simulation uniformly. Every simulation's state stays resident on
the device (vd_server); admission is bounded by an HBM budget.

Frame contents come from per-(L, recipe) pools of `pool` consecutive frames
on the device (simulations of the same kind start at different pool
offsets), so generating inputs does not dominate the run; the RSA recipe
uses a capped rejection budget here (20k consecutive rejections).

``run`` replays one arrival trace through the server with batching
(`max_batch` simulations per step). ``run_plain`` replays it through the plain
per-frame path: one vd_push_frame context per simulation, all on one stream,
frames pushed one at a time in arrival order (FIFO). Both stamp each frame
with its arrival time (trace start + the trace's offset, on the library's
clock) and report frames/s, Gsites/s and the p50/p99 of completion - arrival,
so host delay before a frame is handed over counts in its latency.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs

SIZES = (512, 1024, 2048, 4096)


def make_pools(Ls, n_frames: int, seed: int = 11, rsa_cap: int = 20000):
    """dict (L, recipe) -> list of float32 host frames."""
    pools = {}
    for L in sorted(set(Ls)):
        pools[(L, "noise")] = list(inputs.noise_frames(L, 4.0, n_frames, 0.005, seed + L))
        pools[(L, "discs")] = [F for F, _ in inputs.disc_frames(L, n_frames, seed + 3 * L,
                                                                  max_consecutive_rejections=rsa_cap)]
    return pools


def poisson_trace(n_sims: int, rate: float, duration: float, seed: int = 7):
    """(arrival time s, sim) pairs of one Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append((t, int(rng.integers(n_sims))))
    return out


def _summary(lat_ms, done_sites, wall, steps, resident_gb, max_batch):
    lat = np.array(lat_ms)
    return {"frames": len(lat), "frames_per_s": len(lat) / wall, "gsites_per_s": done_sites / wall / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "steps": steps, "resident_gb": resident_gb, "wall_s": wall,
            "max_batch": max_batch}


def run(sims, dev_pools, trace, max_batch: int, budget_bytes: int, stream=None, frame_check=None):
    """Replay `trace` through a vd_server; returns a dict of measurements.

    sims: list of (L, recipe); dev_pools: (L, recipe) -> list of device tensors.
    frame_check: optional callable(server, done tuple) called for every
    finished frame (the server then keeps per-frame change lists).
    """
    import torch

    from . import vd

    stream = stream or torch.cuda.current_stream()
    sv = vd.Server([(L, L) for L, _ in sims], budget_bytes=budget_bytes, max_batch=max_batch,
                   stream=stream.cuda_stream, keep_changes=frame_check is not None)
    count = [0] * len(sims)
    lat = []
    done_sites = 0
    torch.cuda.synchronize()
    t0 = vd.clock_ns()
    i = 0
    last_done = None

    def retire(ds):
        nonlocal done_sites, last_done
        for d in ds:
            ticket, s, status, ta, ts, td = d[:6]
            if status != 0:
                raise RuntimeError(f"frame of sim {s} failed: {vd.status_string(status)}")
            lat.append((td - ta) / 1e6)
            done_sites += sims[s][0] ** 2
            last_done = td
            if frame_check is not None:
                frame_check(sv, d)

    while i < len(trace) or sv.stats()["frames_done"] < len(trace):
        now = vd.clock_ns()
        while i < len(trace) and t0 + int(trace[i][0] * 1e9) <= now:
            s = trace[i][1]
            L, rec = sims[s]
            pool = dev_pools[(L, rec)]
            sv.submit(s, pool[(count[s] + s) % len(pool)], t0 + int(trace[i][0] * 1e9))
            count[s] += 1
            i += 1
        retire(sv.poll(wait=False))
        if i >= len(trace):
            retire(sv.poll(wait=True))
    st = sv.stats()
    sv.close()
    wall = (last_done - (t0 + int(trace[0][0] * 1e9))) / 1e9
    return _summary(lat, done_sites, wall, st["steps"], st["resident_bytes"] / 1e9, max_batch)


def run_plain(sims, dev_pools, trace, stream=None):
    """The plain per-frame path on the same trace: one context per simulation
    (its state resident), every frame pushed with vd_push_frame on one stream
    in arrival order, completion seen through a CUDA event per frame."""
    import collections

    import torch

    from . import vd

    stream = stream or torch.cuda.current_stream()
    dets = [vd.Detector(L, L, stream=stream.cuda_stream) for L, _ in sims]
    count = [0] * len(sims)
    lat = []
    done_sites = 0
    pending = collections.deque()
    events = [torch.cuda.Event() for _ in range(64)]
    torch.cuda.synchronize()
    t0 = vd.clock_ns()
    i = 0
    k = 0
    last_done = None
    while i < len(trace) or pending:
        now = vd.clock_ns()
        while i < len(trace) and t0 + int(trace[i][0] * 1e9) <= now and len(pending) < len(events):
            s = trace[i][1]
            L, rec = sims[s]
            pool = dev_pools[(L, rec)]
            dets[s].push(pool[(count[s] + s) % len(pool)])
            ev = events[k % len(events)]
            k += 1
            ev.record(stream)
            pending.append((t0 + int(trace[i][0] * 1e9), ev, s))
            count[s] += 1
            i += 1
        while pending and pending[0][1].query():
            ta, _, s = pending.popleft()
            td = vd.clock_ns()
            lat.append((td - ta) / 1e6)
            done_sites += sims[s][0] ** 2
            last_done = td
    for d in dets:
        d.close()
    wall = (last_done - (t0 + int(trace[0][0] * 1e9))) / 1e9
    return _summary(lat, done_sites, wall, len(trace), 0.0, 1)


def serve_workload(n_sims: int = 64, rate: float = 2000.0, duration: float = 5.0, pool: int = 4,
                   budget_gb: float = 40.0, seed: int = 5):
    """Build the served workload and measure batched vs one-frame-per-step."""
    import torch

    params = inputs.serve_sims(n_sims, seed)
    sims = [(L, rec) for L, rec, _ in params]
    host_pools = make_pools([L for L, _ in sims], pool)
    dev_pools = {k: [torch.from_numpy(F).cuda() for F in v] for k, v in host_pools.items()}
    trace = poisson_trace(n_sims, rate, duration, seed)
    budget = int(budget_gb * 1e9)
    served = run(sims, dev_pools, trace, max_batch=n_sims, budget_bytes=budget)
    plain = run_plain(sims, dev_pools, trace)
    offered = sum(sims[s][0] ** 2 for _, s in trace) / duration / 1e9
    return {"served": served, "plain": plain, "offered_gsites_per_s": offered, "arrivals": len(trace),
            "sims": n_sims, "rate": rate, "duration_s": duration}
