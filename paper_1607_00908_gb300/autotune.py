"""Autotuner of the launch shapes of a batch (vd_batch_set_tuning).

The graph stage's form (one block per instance, or grid-wide kernels), the
owner kernel's patch layout, the bucket side of the centre grid (a fraction
of the mean centre spacing) and the reach of the owner search's first round
change only the speed: every setting gives bit-identical results.
The best setting depends on the lattice size and the density of bubbles, so
the tuner times candidates on the batch's own frames and keeps the fastest
per (lattice-size class, density class) in a JSON cache (path from
VD_AUTOTUNE_CACHE, default ~/.cache/vd_autotune.json).

Candidates are searched one parameter at a time (graph-stage form, patch
layout, bucket side, first reach), each timed as whole pushes with CUDA events on the
batch's stream after a warm-up push (the best of three rounds); a candidate
replaces the current setting only when it is faster by more than 1%, so that
timing noise does not pick among equal settings. Timing pushes advance the batch: tune it
on the first frames of a run, before the frames whose results are used.
"""
from __future__ import annotations

import json
import math
import os

from . import vd

PATCHES = (vd.VD_PATCH_8x8, vd.VD_PATCH_16x8, vd.VD_PATCH_16x16, vd.VD_PATCH_32x8)
BUCKETS = (50, 70, 100, 140)
RINGS = (0, 9, 24)
GRAPH = (1, 0)
DEFAULT = dict(voronoi_patch=vd.VD_PATCH_8x8, bucket_pct=100, ring0=9)


def cache_path() -> str:
    return os.environ.get("VD_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "vd_autotune.json"))


def key_of(sizes, bubbles) -> str:
    """(lattice-size class, density class): log2 of the mean sites per lattice
    and log2 of the sites per bubble, rounded."""
    sites = [lx * ly for lx, ly in sizes]
    mean = sum(sites) / len(sites)
    dens = sum(sites) / max(1, sum(bubbles))
    return f"L{round(math.log2(mean))}_s{round(math.log2(max(dens, 1.0)))}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_push(b, fields, stream, reps: int, rounds: int = 3) -> float:
    """ms per push: the best of `rounds` rounds of `reps` pushes (the best
    round is the least disturbed by other work on the device)."""
    import torch
    b.push(fields)   # warm-up (and graph capture after a change of layout)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(rounds):
        e0.record(stream)
        for _ in range(reps):
            b.push(fields)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / reps)
    return best


def tune(b, fields, stream, reps: int = 8, use_cache: bool = True) -> dict:
    """Pick and set the fastest tuning of batch `b` (a vd.Batch) for pushes of
    `fields` (its device frames); returns the chosen setting with its key,
    the ms per push of the default and of the chosen setting, and whether it
    came from the cache."""
    b.push(fields)
    bubbles = [b.counts(i)[0] for i in range(len(b.sizes))]
    key = key_of(b.sizes, bubbles)
    path = cache_path()
    cache = _load(path) if use_cache else {}
    if key in cache:
        t = cache[key]
        b.set_tuning(t["voronoi_patch"], t["bucket_pct"], t["ring0"], t.get("graph_blocks"))
        return dict(t, key=key, cached=True)
    # the batch's own default graph-stage form (by lattice size) is the start
    cur = dict(DEFAULT, graph_blocks=b.tuning()["graph_blocks"])
    b.set_tuning(**cur)
    base = best_ms = _time_push(b, fields, stream, reps)
    tried = {tuple(cur.values()): base}
    for name, values in (("graph_blocks", GRAPH), ("voronoi_patch", PATCHES), ("bucket_pct", BUCKETS),
                         ("ring0", RINGS)):
        for v in values:
            cand = dict(cur, **{name: v})
            k = tuple(cand.values())
            if k in tried:
                continue
            b.set_tuning(**cand)
            tried[k] = ms = _time_push(b, fields, stream, reps)
            if ms < 0.99 * best_ms:
                best_ms, cur = ms, cand
        b.set_tuning(**cur)
    result = dict(cur, default_ms=base, tuned_ms=best_ms, candidates=len(tried))
    if use_cache:
        cache = _load(path)
        cache[key] = result
        _store(path, cache)
    b.set_tuning(**cur)
    return dict(result, key=key, cached=False)
