"""Served form (vd_server_*): continuous batching gives each simulation
exactly the results it gets alone.

Frames of several simulations are submitted in an interleaved, seeded order
while earlier steps are still on the device; every finished frame's counts
(bubbles, links, breaking, arising) and every simulation's final labels and
flip lists must equal those of the same frame sequence pushed through its
own vd_push_frame context.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import serve  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402
from tests.oracle_digest import array_digest, oracle_sequence  # noqa: E402

FULL = os.environ.get("VD_FULL", "0") == "1"


def _setup(seed=3):
    sizes = [(96, 96), (128, 80), (200, 200), (64, 64), (160, 120)]
    n_frames = 5
    frames = []
    for k, (lx, ly) in enumerate(sizes):
        seq = list(I.noise_frames(ly, 2.5 + 0.5 * k, n_frames, 0.03, seed + k, Lx=lx))
        frames.append([torch.from_numpy(F).cuda() for F in seq])
    rng = np.random.default_rng(seed)
    order = []
    for f in range(n_frames):
        sims = list(rng.permutation(len(sizes)))
        order += [(s, f) for s in sims]
    return sizes, frames, order


def _alone_counts(sizes, frames):
    out = {}
    finals = {}
    for s, (lx, ly) in enumerate(sizes):
        det = vd.Detector(lx, ly)
        for f, F in enumerate(frames[s]):
            det.push(F)
            ch = det.changes()
            out[(s, f)] = (ch["K"], ch["n_edges"], len(ch["breaking"]), len(ch["arising"]))
        finals[s] = (det.labels(), det.changes())
        det.close()
    return out, finals


@pytest.mark.parametrize("max_batch,budget_extra", [(5, 1 << 30), (3, 1 << 30), (5, 300_000)])
def test_served_results_equal_alone(max_batch, budget_extra):
    sizes, frames, order = _setup()
    want, finals = _alone_counts(sizes, frames)
    # resident state measured by a first server; the budget leaves room for
    # `budget_extra` bytes of frames in flight
    probe = vd.Server(sizes, budget_bytes=1 << 40, max_batch=max_batch)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    sv = vd.Server(sizes, budget_bytes=resident + budget_extra, max_batch=max_batch)
    seen = {}
    pos = [0] * len(sizes)
    tickets = {}
    for s, f in order:
        tickets[sv.submit(s, frames[s][f])] = (s, f)
        for d in sv.poll(wait=False):
            seen[tickets[d[0]]] = d
    while len(seen) < len(order):
        for d in sv.poll(wait=True):
            seen[tickets[d[0]]] = d
    st = sv.stats()
    assert st["frames_done"] == len(order)
    for key, d in seen.items():
        ticket, s, status, ts, td, K, E, nb, na = d
        assert status == 0
        assert (K, E, nb, na) == want[key], (key, (K, E, nb, na), want[key])
        assert td >= ts
    for s in range(len(sizes)):
        lab, ch = finals[s]
        assert np.array_equal(sv.labels(s), lab)
        got = sv.changes(s)
        assert np.array_equal(got["breaking"], ch["breaking"]) and np.array_equal(got["arising"], ch["arising"])
    if max_batch > 1 and budget_extra > 1 << 20:
        assert st["steps"] < len(order)     # frames were batched
    sv.close()


def test_budget_below_resident_state_is_refused():
    with pytest.raises(vd.VdError) as e:
        vd.Server([(256, 256)], budget_bytes=1 << 20, max_batch=4)
    assert e.value.status == vd.VD_ERR_CAPACITY


def test_small_served_workload_runs():
    """The served driver on a reduced trace: batched and one-at-a-time both
    finish every frame; batching takes fewer steps."""
    sims = [(256, "noise"), (256, "discs"), (512, "noise"), (512, "discs")]
    pools = serve.make_pools([256, 512], 3, rsa_cap=2000)
    dev = {k: [torch.from_numpy(F).cuda() for F in v] for k, v in pools.items()}
    trace = serve.poisson_trace(len(sims), rate=400.0, duration=0.5, seed=2)
    a = serve.run(sims, dev, trace, max_batch=4, budget_bytes=8 << 30)
    b = serve.run(sims, dev, trace, max_batch=1, budget_bytes=8 << 30)
    assert a["frames"] == b["frames"] == len(trace)
    assert a["steps"] <= b["steps"]


def test_served_options_equal_alone():
    """Simulations with different options (event classes, centre match,
    8-connectivity, the vertex link rule, walls) served together: every
    simulation's final labels, flip lists and event flags equal those of its
    own vd_push_frame context with the same options."""
    sizes, frames, order = _setup(seed=7)
    opts = [dict(events=True), dict(events=True, match_rule=vd.VD_MATCH_CENTROID, match_radius=4),
            dict(connectivity=8), dict(edge_rule=vd.VD_EDGE_VERTEX), dict(walls=vd.VD_WALL_X, events=True)]
    finals = {}
    for s, (lx, ly) in enumerate(sizes):
        det = vd.Detector(lx, ly, **opts[s])
        for F in frames[s]:
            det.push(F)
        finals[s] = (det.labels(), det.changes())
        det.close()
    sv = vd.Server(sizes, budget_bytes=1 << 40, max_batch=4, options=opts)
    for s, f in order:
        sv.submit(s, frames[s][f])
    done = 0
    while done < len(order):
        done += len(sv.poll(wait=True))
    for s in range(len(sizes)):
        lab, ch = finals[s]
        assert np.array_equal(sv.labels(s), lab), s
        got = sv.changes(s)
        assert np.array_equal(got["breaking"], ch["breaking"]), s
        assert np.array_equal(got["arising"], ch["arising"]), s
        assert np.array_equal(got["active"], ch["active"]), s
    sv.close()


@pytest.mark.skipif(not FULL, reason="the full served workload takes minutes of oracle time: VD_FULL=1")
def test_served_workload_full_size():
    """The served workload's 64 simulations (512^2 ... 4096^2, smoothed noise
    and droplets) on a seeded Poisson trace of 500 arrivals, frames taken
    from the shared pools in the served driver's order: every simulation's
    per-frame counts and final labels and flip lists equal those run alone,
    and for the first 8 simulations those of the oracle."""
    import multiprocessing as mp
    params = I.serve_sims()
    sims = [(L, rec) for L, rec, _ in params]
    host_pools = serve.make_pools([L for L, _ in sims], 4)
    trace = serve.poisson_trace(len(sims), 2000.0, 0.25, 5)
    seqs = [[] for _ in sims]
    for _, s in trace:
        seqs[s].append((len(seqs[s]) + s) % 4)
    tasks = [(sims[s][0], host_pools[sims[s]], seqs[s]) for s in range(8)]
    with mp.get_context("spawn").Pool(8) as pool:
        oracle = pool.map(oracle_sequence, tasks)
    dev_pools = {k: [torch.from_numpy(F).cuda() for F in v] for k, v in host_pools.items()}
    del host_pools
    # alone: one context per simulation
    alone, finals = {}, {}
    for s, (L, rec) in enumerate(sims):
        det = vd.Detector(L, L)
        for k, j in enumerate(seqs[s]):
            det.push(dev_pools[(L, rec)][j])
            ch = det.changes()
            alone[(s, k)] = (ch["K"], ch["n_edges"], len(ch["breaking"]), len(ch["arising"]))
        if seqs[s]:
            finals[s] = (det.labels(), det.changes())
        det.close()
    # served, in trace order
    sv = vd.Server([(L, L) for L, _ in sims], budget_bytes=40_000_000_000, max_batch=len(sims))
    tickets, seen, count = {}, {}, [0] * len(sims)
    for _, s in trace:
        L, rec = sims[s]
        tickets[sv.submit(s, dev_pools[(L, rec)][seqs[s][count[s]]])] = (s, count[s])
        count[s] += 1
        for d in sv.poll(wait=False):
            seen[tickets[d[0]]] = d
    while len(seen) < len(trace):
        for d in sv.poll(wait=True):
            seen[tickets[d[0]]] = d
    for key, d in seen.items():
        ticket, s, status, ts, td, K, E, nb, na = d
        assert status == 0, key
        assert (K, E, nb, na) == alone[key], (key, (K, E, nb, na), alone[key])
    for s, (lab, ch) in finals.items():
        assert np.array_equal(sv.labels(s), lab), s
        got = sv.changes(s)
        assert np.array_equal(got["breaking"], ch["breaking"]) and np.array_equal(got["arising"], ch["arising"]), s
    for s in range(8):
        counts, lab_digest, breaking, arising = oracle[s]
        assert [alone[(s, k)] for k in range(len(seqs[s]))] == counts, s
        if seqs[s]:
            assert array_digest(finals[s][0]) == lab_digest, s
            assert np.array_equal(finals[s][1]["breaking"], breaking), s
            assert np.array_equal(finals[s][1]["arising"], arising), s
    sv.close()
