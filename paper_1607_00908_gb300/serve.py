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
(`max_batch` simulations per step) or without (`max_batch=1`: one frame per
step, first come first served) and reports frames/s, Gsites/s and the
p50/p99 of completion - arrival per frame.
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


def run(sims, dev_pools, trace, max_batch: int, budget_bytes: int, stream=None):
    """Replay `trace` through a vd_server; returns a dict of measurements.

    sims: list of (L, recipe); dev_pools: (L, recipe) -> list of device tensors.
    """
    import torch

    from . import vd

    stream = stream or torch.cuda.current_stream()
    sv = vd.Server([(L, L) for L, _ in sims], budget_bytes=budget_bytes, max_batch=max_batch,
                   stream=stream.cuda_stream)
    count = [0] * len(sims)
    lat = []
    done_sites = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    i = 0
    first_submit = None
    last_done = None
    while i < len(trace) or sv.stats()["frames_done"] < len(trace):
        now = time.perf_counter() - t0
        while i < len(trace) and trace[i][0] <= now:
            s = trace[i][1]
            L, rec = sims[s]
            pool = dev_pools[(L, rec)]
            sv.submit(s, pool[(count[s] + s) % len(pool)])
            count[s] += 1
            if first_submit is None:
                first_submit = time.perf_counter()
            i += 1
        for ticket, s, status, ts, td, *_ in sv.poll(wait=False):
            if status != 0:
                raise RuntimeError(f"frame of sim {s} failed: {vd.status_string(status)}")
            lat.append((td - ts) / 1e6)
            done_sites += sims[s][0] ** 2
            last_done = time.perf_counter()
        if i >= len(trace):
            for ticket, s, status, ts, td, *_ in sv.poll(wait=True):
                lat.append((td - ts) / 1e6)
                done_sites += sims[s][0] ** 2
                last_done = time.perf_counter()
    st = sv.stats()
    sv.close()
    wall = last_done - first_submit
    lat = np.array(lat)
    return {"frames": len(lat), "frames_per_s": len(lat) / wall, "gsites_per_s": done_sites / wall / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "steps": st["steps"], "resident_gb": st["resident_bytes"] / 1e9,
            "wall_s": wall, "max_batch": max_batch}


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
    plain = run(sims, dev_pools, trace, max_batch=1, budget_bytes=budget)
    offered = sum(sims[s][0] ** 2 for _, s in trace) / duration / 1e9
    return {"served": served, "plain": plain, "offered_gsites_per_s": offered, "arrivals": len(trace),
            "sims": n_sims, "rate": rate, "duration_s": duration}
