"""Served form (vd_server_*): continuous batching gives each simulation
exactly the results it gets alone.

Frames of several simulations are submitted in an interleaved, seeded order
while earlier steps are still on the device; every finished frame's breaking
and arising lists, past keys and active flags (kept per frame by the server)
and every simulation's final labels must equal those of the same frame
sequence pushed through its own vd_push_frame context. Simulations are also
opened and closed while others run.
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


def _alone_changes(sizes, frames, options=None):
    """Every frame's changes and the final labels of each simulation run alone."""
    out = {}
    finals = {}
    for s, (lx, ly) in enumerate(sizes):
        det = vd.Detector(lx, ly, **((options or {}).get(s, {})))
        for f, F in enumerate(frames[s]):
            det.push(F)
            out[(s, f)] = det.changes()
        finals[s] = (det.labels(), det.changes())
        det.close()
    return out, finals


def _same_frame(got, want, tag):
    for k in ("K", "n_edges", "K_prev", "n_matched", "global_trigger"):
        assert got[k] == want[k], (tag, k, got[k], want[k])
    for k in ("breaking", "breaking_prev", "arising", "active"):
        assert np.array_equal(got[k], want[k]), (tag, k)


def _drain(sv, tickets, seen, want):
    """Poll once more; compare every retired frame with its alone result."""
    for d in sv.poll(wait=True):
        _check_done(sv, d, tickets, seen, want)


def _check_done(sv, d, tickets, seen, want):
    ticket, s, status, ta, ts, td, K, E, nb, na = d
    key = tickets[ticket]
    assert status == 0, key
    assert td >= ts >= ta > 0, key
    w = want[key]
    assert (K, E, nb, na) == (w["K"], w["n_edges"], len(w["breaking"]), len(w["arising"])), key
    _same_frame(sv.frame_changes(ticket, K), w, key)
    seen[key] = d


@pytest.mark.parametrize("max_batch,budget_extra", [(5, 1 << 30), (3, 1 << 30), (5, 300_000)])
def test_served_results_equal_alone(max_batch, budget_extra):
    sizes, frames, order = _setup()
    want, finals = _alone_changes(sizes, frames)
    # resident state measured by a first server; the budget leaves room for
    # `budget_extra` bytes of frames in flight
    probe = vd.Server(sizes, budget_bytes=1 << 40, max_batch=max_batch)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    sv = vd.Server(sizes, budget_bytes=resident + budget_extra, max_batch=max_batch, keep_changes=True)
    seen = {}
    tickets = {}
    for s, f in order:
        tickets[sv.submit(s, frames[s][f], vd.clock_ns())] = (s, f)
        for d in sv.poll(wait=False):
            _check_done(sv, d, tickets, seen, want)
    while len(seen) < len(order):
        _drain(sv, tickets, seen, want)
    st = sv.stats()
    assert st["frames_done"] == len(order)
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


def test_simulations_opened_and_closed_while_others_run():
    """Three simulations start; two more are opened after the first frames
    are queued (one of them refused first by a budget that cannot hold it);
    one simulation is closed once drained and its id is refused afterwards.
    Every frame of every simulation equals its alone run, element by element."""
    sizes, frames, order = _setup(seed=11)
    want, finals = _alone_changes(sizes, frames)
    first = [0, 1, 2]
    probe = vd.Server([sizes[s] for s in first], budget_bytes=1 << 40, max_batch=8)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    # room for the frames in flight (at most 5 x 160 KB) but not for another
    # lattice's resident state (several MB even at 64 x 64)
    sv = vd.Server([sizes[s] for s in first], budget_bytes=resident + (2 << 20), max_batch=8, keep_changes=True)
    ids = {s: s for s in first}          # workload sim -> server id
    tickets, seen = {}, {}
    pending = [(s, f) for s, f in order]
    # the first two frames of the three open simulations
    for s, f in [p for p in pending if p[0] in first and p[1] < 2]:
        tickets[sv.submit(ids[s], frames[s][f], vd.clock_ns())] = (s, f)
    for d in sv.poll(wait=False):
        _check_done(sv, d, tickets, seen, want)
    # a 200 x 200 simulation does not fit the remaining budget
    with pytest.raises(vd.VdError) as e:
        sv.open_sim(sizes[2])
    assert e.value.status == vd.VD_ERR_CAPACITY
    sv.close()
    # a server with room for the newcomers, which join while frames are in flight
    sv = vd.Server([sizes[s] for s in first], budget_bytes=1 << 40, max_batch=8, keep_changes=True)
    tickets, seen = {}, {}
    for s, f in [p for p in pending if p[0] in first and p[1] < 2]:
        tickets[sv.submit(ids[s], frames[s][f], vd.clock_ns())] = (s, f)
    for d in sv.poll(wait=False):
        _check_done(sv, d, tickets, seen, want)
    for s in (3, 4):
        ids[s] = sv.open_sim(sizes[s])
    assert ids[3] == 3 and ids[4] == 4
    rest = [p for p in pending if not (p[0] in first and p[1] < 2)]
    for s, f in rest:
        tickets[sv.submit(ids[s], frames[s][f], vd.clock_ns())] = (s, f)
        for d in sv.poll(wait=False):
            _check_done(sv, d, tickets, seen, want)
    while len(seen) < len(order):
        _drain(sv, tickets, seen, want)
    # simulation 1 is drained: close it; its id is refused afterwards
    lab1 = sv.labels(ids[1])
    assert np.array_equal(lab1, finals[1][0])
    sv.close_sim(ids[1])
    with pytest.raises(vd.VdError) as e:
        sv.submit(ids[1], frames[1][0])
    assert e.value.status == vd.VD_ERR_INVALID
    with pytest.raises(vd.VdError) as e:
        sv.labels(ids[1])
    assert e.value.status == vd.VD_ERR_INVALID
    for s in (0, 2, 3, 4):
        assert np.array_equal(sv.labels(ids[s]), finals[s][0]), s
    # a simulation opened alone leaves the budget when closed
    before = sv.stats()["resident_bytes"]
    sid = sv.open_sim((64, 64))
    assert sv.stats()["resident_bytes"] > before
    sv.close_sim(sid)
    assert sv.stats()["resident_bytes"] == before
    sv.close()


def test_served_checkpoint_moves_a_simulation():
    """A simulation's state exported from one server and imported into a
    simulation of another continues with the same changes as alone."""
    sizes, frames, order = _setup(seed=13)
    want, _ = _alone_changes(sizes, frames)
    a = vd.Server(sizes, budget_bytes=1 << 40, max_batch=8)
    for f in range(2):
        for s in range(len(sizes)):
            a.submit(s, frames[s][f])
    n = 0
    while n < 2 * len(sizes):
        n += len(a.poll(wait=True))
    blob = a.export_state(2)
    a.close()
    b = vd.Server([], budget_bytes=1 << 40, max_batch=8, keep_changes=True)
    sid = b.open_sim(sizes[2])
    b.import_state(sid, blob)
    for f in range(2, len(frames[2])):
        t = b.submit(sid, frames[2][f])
        ds = b.poll(wait=True)
        assert [d[0] for d in ds] == [t]
        _same_frame(b.frame_changes(t, ds[0][6]), want[(2, f)], ("moved", f))
    b.close()


def test_small_served_workload_runs():
    """The served driver on a reduced trace: batched and one-at-a-time both
    finish every frame; batching takes fewer steps."""
    sims = [(256, "noise"), (256, "discs"), (512, "noise"), (512, "discs")]
    pools = serve.make_pools([256, 512], 3, rsa_cap=2000)
    dev = {k: [torch.from_numpy(F).cuda() for F in v] for k, v in pools.items()}
    trace = serve.poisson_trace(len(sims), rate=400.0, duration=0.5, seed=2)
    a = serve.run(sims, dev, trace, max_batch=4, budget_bytes=8 << 30)
    b = serve.run(sims, dev, trace, max_batch=1, budget_bytes=8 << 30)
    c = serve.run_plain(sims, dev, trace)
    assert a["frames"] == b["frames"] == c["frames"] == len(trace)
    assert a["steps"] <= b["steps"]
    for r in (a, b, c):
        assert 0 < r["p50_ms"] <= r["p99_ms"]


def test_served_options_equal_alone():
    """Simulations with different options (event classes, centre match,
    8-connectivity, the vertex link rule, walls) served together: every
    simulation's final labels, flip lists and event flags equal those of its
    own vd_push_frame context with the same options."""
    sizes, frames, order = _setup(seed=7)
    opts = [dict(events=True), dict(events=True, match_rule=vd.VD_MATCH_CENTROID, match_radius=4),
            dict(connectivity=8), dict(edge_rule=vd.VD_EDGE_VERTEX), dict(walls=vd.VD_WALL_X, events=True)]
    want, finals = _alone_changes(sizes, frames, dict(enumerate(opts)))
    sv = vd.Server(sizes, budget_bytes=1 << 40, max_batch=4, options=opts, keep_changes=True)
    tickets, seen = {}, {}
    for s, f in order:
        tickets[sv.submit(s, frames[s][f])] = (s, f)
    while len(seen) < len(order):
        _drain(sv, tickets, seen, want)
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
    from the shared pools in the served driver's order: every frame of every
    simulation equals the same frame run alone, element by element (breaking
    and arising lists, past keys, active flags), final labels too; and every
    frame of the first 8 simulations equals the oracle's."""
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
            alone[(s, k)] = det.changes()
        if seqs[s]:
            finals[s] = det.labels()
        det.close()
    # served, in trace order, every retired frame compared as it retires
    sv = vd.Server([(L, L) for L, _ in sims], budget_bytes=40_000_000_000, max_batch=len(sims), keep_changes=True)
    tickets, seen, count = {}, {}, [0] * len(sims)
    for _, s in trace:
        L, rec = sims[s]
        tickets[sv.submit(s, dev_pools[(L, rec)][seqs[s][count[s]]], vd.clock_ns())] = (s, count[s])
        count[s] += 1
        for d in sv.poll(wait=False):
            _check_done(sv, d, tickets, seen, alone)
    while len(seen) < len(trace):
        _drain(sv, tickets, seen, alone)
    for s, lab in finals.items():
        assert np.array_equal(sv.labels(s), lab), s
    for s in range(8):
        frames_o, lab_digest = oracle[s]
        assert len(frames_o) == len(seqs[s])
        for k, r in enumerate(frames_o):
            a = alone[(s, k)]
            assert (a["K"], a["n_edges"]) == (r["K"], r["E"]), (s, k)
            for key in ("breaking", "breaking_prev", "arising", "active"):
                assert np.array_equal(a[key], r[key]), (s, k, key)
        if seqs[s]:
            assert array_digest(finals[s]) == lab_digest, s
    sv.close()
