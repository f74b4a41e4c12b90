"""GPU parity of the batched forms against the CPU oracle (exact).

* Batch of lattices of uneven sizes advanced together (vd_batch_push).
* Frame sequence (vd_batch_create_sequence): n consecutive frames per push,
  instance i's past frame is instance i-1 of the same push.
* Subsets of a batch advancing at different times (vd_batch_push_subset),
  the mechanism the served form uses, and equality of every result with the
  same lattice run alone.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402
from tests.oracle_digest import batched_frames, oracle_digests, site_digests  # noqa: E402

FULL = os.environ.get("VD_FULL", "0") == "1"


def check(b, i, r, tag):
    K, E, _ = b.counts(i)
    assert K == r["K"], (tag, K, r["K"])
    assert np.array_equal(b.labels(i), r["labels"]), f"{tag} labels"
    assert np.array_equal(b.centroids(i), r["centroids"]), f"{tag} centroids"
    assert np.array_equal(b.owners(i), r["owners"]), f"{tag} owners"
    assert np.array_equal(b.edges(i), r["edges"]), f"{tag} edges"
    ch = b.changes(i)
    assert ch["K_prev"] == r["K_prev"], (tag, ch["K_prev"], r["K_prev"])
    assert ch["n_matched"] == r["n_matched"], (tag, ch["n_matched"], r["n_matched"])
    assert np.array_equal(ch["breaking"], r["breaking"]), f"{tag} breaking"
    assert np.array_equal(ch["breaking_prev"], r["breaking_prev"]), f"{tag} breaking_prev"
    assert np.array_equal(ch["arising"], r["arising"]), f"{tag} arising"
    assert np.array_equal(ch["active"], r["active"]), f"{tag} active"


def frames_for(L, sigma, seed, n, Lx=None):
    return list(I.noise_frames(L, sigma, n, 0.03, seed, Lx=Lx))


def test_uneven_batch_matches_per_instance_oracle():
    specs = [(64, 64, 2.0), (96, 70, 3.0), (130, 130, 2.5), (200, 150, 4.0), (257, 257, 3.0), (33, 200, 2.0)]
    n_frames = 3
    seqs = [frames_for(ly, s, 10 + k, n_frames, Lx=lx) for k, (lx, ly, s) in enumerate(specs)]
    b = vd.Batch([(lx, ly) for lx, ly, _ in specs])
    refs = [O.Detector(lx, ly, voronoi="brute") for lx, ly, _ in specs]
    for f in range(n_frames):
        dev = [torch.from_numpy(seq[f]).cuda() for seq in seqs]
        b.push(dev)
        for i, ref in enumerate(refs):
            check(b, i, ref.push(seqs[i][f]), f"inst {i} frame {f}")
    b.close()


@pytest.mark.parametrize("n_seq,pushes", [(4, 3), (1, 3), (7, 2)])
def test_frame_sequence_matches_oracle(n_seq, pushes):
    L = 150
    frames = frames_for(L, 3.0, 77, n_seq * pushes)
    b = vd.Batch([(L, L)], sequence=n_seq)
    ref = O.Detector(L, L, voronoi="brute")
    for p in range(pushes):
        chunk = frames[p * n_seq:(p + 1) * n_seq]
        b.push([torch.from_numpy(F).cuda() for F in chunk])
        for i, F in enumerate(chunk):
            r = ref.push(F)
            check(b, i, r, f"push {p} frame {i}")
            assert b.changes(i)["frame"] == p * n_seq + i
    b.close()


def test_subsets_and_alone_vs_mix():
    """Instances advanced at different times give exactly the results each
    lattice gets when run alone with vd_push_frame."""
    specs = [(80, 80), (120, 90), (64, 130)]
    seqs = [frames_for(ly, 3.0, 200 + k, 4, Lx=lx) for k, (lx, ly) in enumerate(specs)]
    b = vd.Batch(specs)
    alone = [vd.Detector(lx, ly) for lx, ly in specs]
    refs = [O.Detector(lx, ly, voronoi="brute") for lx, ly in specs]
    pos = [0, 0, 0]
    schedule = [[0, 2], [1], [0, 1, 2], [2, 0], [1, 0], [1], [2]]
    for act in schedule:
        dev = [torch.from_numpy(seqs[i][pos[i]]).cuda() for i in act]
        b.push_subset(act, dev)
        for i, d in zip(act, dev):
            alone[i].push(d)
            r = refs[i].push(seqs[i][pos[i]])
            check(b, i, r, f"subset inst {i} frame {pos[i]}")
            assert np.array_equal(b.labels(i), alone[i].labels())
            assert np.array_equal(b.owners(i), alone[i].owners())
            ca, cb = b.changes(i), alone[i].changes()
            assert np.array_equal(ca["breaking"], cb["breaking"]) and np.array_equal(ca["arising"], cb["arising"])
            pos[i] += 1
    b.close()
    for d in alone:
        d.close()


def _pinned(frames):
    return [torch.from_numpy(np.ascontiguousarray(F)).pin_memory() for F in frames]


def test_staged_host_pipeline_and_packed_changes_match_oracle():
    """Host frames staged on the copy stream while the previous push runs
    (vd_batch_stage_host / vd_batch_push_staged), results read packed for the
    whole sequence (vd_batch_get_changes_all): every frame equals the oracle
    and the per-frame getters."""
    L, n_seq, pushes = 140, 5, 4
    frames = frames_for(L, 3.0, 41, n_seq * pushes)
    host = [_pinned(frames[p * n_seq:(p + 1) * n_seq]) for p in range(pushes)]
    b = vd.Batch([(L, L)], sequence=n_seq)
    ref = O.Detector(L, L, voronoi="brute")
    b.stage_host_ptrs([h.data_ptr() for h in host[0]])
    b.push_staged()
    for p in range(pushes):
        if p + 1 < pushes:   # next frames copied while this push runs
            b.stage_host_ptrs([h.data_ptr() for h in host[p + 1]])
        allc = b.changes_all()
        ob = oa = ok = 0
        for i in range(n_seq):
            r = ref.push(frames[p * n_seq + i])
            assert allc["status"][i] == vd.VD_OK
            assert allc["n_now"][i] == r["K"] and allc["n_prev"][i] == r["K_prev"]
            nb, na, nk = allc["n_breaking"][i], allc["n_arising"][i], allc["n_now"][i]
            assert np.array_equal(allc["breaking"][ob:ob + nb], r["breaking"]), (p, i)
            assert np.array_equal(allc["breaking_prev"][ob:ob + nb], r["breaking_prev"]), (p, i)
            assert np.array_equal(allc["arising"][oa:oa + na], r["arising"]), (p, i)
            assert np.array_equal(allc["active"][ok:ok + nk], r["active"]), (p, i)
            check(b, i, r, f"push {p} frame {i}")
            ob, oa, ok = ob + nb, oa + na, ok + nk
        assert (ob, oa, ok) == (len(allc["breaking"]), len(allc["arising"]), len(allc["active"]))
        if p + 1 < pushes:
            b.push_staged()
    b.close()


def test_push_staged_needs_a_stage():
    b = vd.Batch([(64, 64)])
    with pytest.raises(vd.VdError) as e:
        b.push_staged()
    assert e.value.status == vd.VD_ERR_STATE
    F = _pinned(frames_for(64, 2.0, 3, 1))
    b.stage_host_ptrs([F[0].data_ptr()])
    b.push_staged()
    with pytest.raises(vd.VdError) as e:
        b.push_staged()
    assert e.value.status == vd.VD_ERR_STATE
    b.close()


def test_staged_uneven_batch_with_a_failing_instance():
    """Uneven batch fed through the staged host path; one instance overflows
    its bubble capacity: vd_batch_get_changes_all reports VD_ERR_CAPACITY for
    it, packs only the others' lists, and those equal the oracle."""
    specs = [(96, 80, 2.5), (64, 64, 0.0), (120, 120, 3.0)]
    n_frames = 3
    cap = 100
    checker = ((np.indices((64, 64)).sum(0) % 2) == 0).astype(np.float32)   # 2048 bubbles > cap
    seqs = []
    for k, (lx, ly, s) in enumerate(specs):
        seqs.append([checker] * n_frames if s == 0.0 else frames_for(ly, s, 60 + k, n_frames, Lx=lx))
    host = [[torch.from_numpy(np.ascontiguousarray(F)).pin_memory() for F in seq] for seq in seqs]
    b = vd.Batch([(lx, ly) for lx, ly, _ in specs], max_components=cap)
    refs = {i: O.Detector(lx, ly, voronoi="brute") for i, (lx, ly, s) in enumerate(specs) if s != 0.0}
    for f in range(n_frames):
        b.stage_host_ptrs([host[i][f].data_ptr() for i in range(len(specs))])
        b.push_staged()
        allc = b.changes_all()
        assert allc["status"][1] == vd.VD_ERR_CAPACITY
        assert allc["n_breaking"][1] == 0 and allc["n_arising"][1] == 0 and allc["n_now"][1] == 0
        ob = oa = ok = 0
        for i, ref in refs.items():
            r = ref.push(seqs[i][f])
            assert allc["status"][i] == vd.VD_OK
            nb, na, nk = allc["n_breaking"][i], allc["n_arising"][i], allc["n_now"][i]
            assert nk == r["K"]
            assert np.array_equal(allc["breaking"][ob:ob + nb], r["breaking"]), (f, i)
            assert np.array_equal(allc["breaking_prev"][ob:ob + nb], r["breaking_prev"]), (f, i)
            assert np.array_equal(allc["arising"][oa:oa + na], r["arising"]), (f, i)
            assert np.array_equal(allc["active"][ok:ok + nk], r["active"]), (f, i)
            check(b, i, r, f"inst {i} frame {f}")
            ob, oa, ok = ob + nb, oa + na, ok + nk
        assert (ob, oa, ok) == (len(allc["breaking"]), len(allc["arising"]), len(allc["active"]))
        with pytest.raises(vd.VdError) as e:
            b.changes(1)
        assert e.value.status == vd.VD_ERR_CAPACITY
    b.close()


def test_batch_with_degenerate_instances():
    """Empty field (no bubble), one bubble covering the whole torus, one
    single-site bubble, and ordinary noise advance in one batch; each equals
    the oracle run alone."""
    L = 48
    empty = np.zeros((L, L), np.float32)
    full = np.ones((L, L), np.float32)
    dot = np.zeros((L, L), np.float32)
    dot[7, 11] = 1.0
    noise = frames_for(L, 2.0, 77, 2)
    seqs = [[empty, empty], [full, full], [dot, dot], noise, [empty, full]]
    b = vd.Batch([(L, L)] * len(seqs))
    refs = [O.Detector(L, L, voronoi="brute") for _ in seqs]
    for f in range(2):
        b.push([torch.from_numpy(np.ascontiguousarray(s[f])).cuda() for s in seqs])
        for i, ref in enumerate(refs):
            check(b, i, ref.push(seqs[i][f]), f"inst {i} frame {f}")
    b.close()



def test_batch_with_mixed_options():
    """One independent batch whose instances differ in every option (event
    classes, centre match, 8-connectivity, the vertex link rule, walls and
    obstacles): each instance's changes equal the oracle run with its own
    options, so the per-instance switches of the shared launches hold."""
    L = 96
    opts = [
        dict(),
        dict(events=True),
        dict(events=True, match_rule=vd.VD_MATCH_CENTROID, match_radius=5),
        dict(connectivity=8),
        dict(edge_rule=vd.VD_EDGE_VERTEX, events=True),
        dict(walls=vd.VD_WALL_X | vd.VD_WALL_Y, events=True),
    ]
    ref_opts = [
        dict(),
        dict(events=True),
        dict(events=True, match="centroid", match_radius=5),
        dict(connectivity=8),
        dict(edge_rule="vertex", events=True),
        dict(walls=(True, True), events=True),
    ]
    n = len(opts)
    seqs = [list(I.noise_frames(L, 2.5 + 0.3 * i, 3, 0.02, 40 + i)) for i in range(n)]
    obst = np.zeros((L, L), dtype=bool)
    obst[10:20, 0:3] = True
    b = vd.Batch([(L, L)] * n, options=opts)
    b.set_obstacles(5, obst)
    refs = [O.Detector(L, L, voronoi="brute", obstacles=obst if i == 5 else None, **ref_opts[i]) for i in range(n)]
    for f in range(3):
        dev = [torch.from_numpy(np.ascontiguousarray(seqs[i][f])).cuda() for i in range(n)]
        b.push(dev)
        for i in range(n):
            r = refs[i].push(seqs[i][f])
            check(b, i, r, f"mixed inst {i} frame {f}")
    b.close()


@pytest.mark.skipif(not FULL, reason="the full batched workload takes minutes of oracle time: VD_FULL=1")
def test_batched_workload_every_instance_and_frame():
    """The batched workload at full size -- 256 instances of 256^2 ... 2048^2
    smoothed noise, 8 frames each, one push per frame -- against the oracle
    for every instance and frame. The oracle runs in spawned worker processes
    (one instance per task) and returns per-site arrays as digests."""
    import multiprocessing as mp
    specs = I.batch_instances()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        want = pool.map(oracle_digests, specs)
    b = vd.Batch([(L, L) for L, _, _ in specs])
    gens = [batched_frames(spec) for spec in specs]
    for f in range(8):
        dev = [torch.from_numpy(next(g)).cuda() for g in gens]
        b.push(dev)
        for i, spec in enumerate(specs):
            w = want[i][f]
            tag = f"instance {i} ({spec[0]}^2) frame {f}"
            K, _, _ = b.counts(i)
            assert K == w["K"], tag
            assert site_digests(b.labels(i), b.owners(i)) == (w["labels"], w["owners"]), tag
            assert np.array_equal(b.centroids(i), w["centroids"]), tag
            assert np.array_equal(b.edges(i), w["edges"]), tag
            ch = b.changes(i)
            for k in ("K_prev", "n_matched"):
                assert ch[k] == w[k], (tag, k)
            for k in ("breaking", "breaking_prev", "arising", "active"):
                assert np.array_equal(ch[k], w[k]), (tag, k)
        del dev
    b.close()


def test_many_instances_and_a_long_sequence():
    """24 uneven lattices in one batch, and a 20-frame sequence pushed twice,
    against the oracle frame by frame."""
    rng = np.random.default_rng(5)
    specs = [(int(rng.integers(40, 97)), int(rng.integers(40, 97)), float(rng.uniform(1.5, 3.5))) for _ in range(24)]
    seqs = [frames_for(ly, s, 200 + k, 2, Lx=lx) for k, (lx, ly, s) in enumerate(specs)]
    b = vd.Batch([(lx, ly) for lx, ly, _ in specs])
    refs = [O.Detector(lx, ly, voronoi="brute") for lx, ly, _ in specs]
    for f in range(2):
        b.push([torch.from_numpy(seq[f]).cuda() for seq in seqs])
        for i, ref in enumerate(refs):
            check(b, i, ref.push(seqs[i][f]), f"inst {i} frame {f}")
    b.close()
    L, n_seq = 80, 20
    frames = frames_for(L, 2.5, 321, 2 * n_seq)
    ref = O.Detector(L, L, voronoi="brute")
    want = [ref.push(F) for F in frames]
    b = vd.Batch([(L, L)], sequence=n_seq)
    dev = [torch.from_numpy(F).cuda() for F in frames]
    for p in range(2):
        b.push(dev[p * n_seq:(p + 1) * n_seq])
        for i in range(n_seq):
            check(b, i, want[p * n_seq + i], f"seq push {p} frame {i}")
    b.close()
