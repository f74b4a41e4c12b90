"""Checkpoint / resume (vd_export_state / vd_import_state).

Section 3.2.3 compares every frame with the previous one, so a detector
carries one frame's state forward: its labels, centroids (with their bucket
grid) and links. A context resumed from an exported state must report
bit-identical changes to the uninterrupted one and to the oracle; a damaged or
foreign blob must be refused without touching the context.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402


def _same_changes(a, b, tag):
    for k in ("K_prev", "K", "n_matched", "n_edges", "global_trigger"):
        assert a[k] == b[k], (tag, k, a[k], b[k])
    for k in ("breaking", "breaking_prev", "arising", "active"):
        assert np.array_equal(a[k], b[k]), (tag, k)


def _oracle_changes_equal(ch, r, tag):
    assert ch["K_prev"] == r["K_prev"] and ch["n_matched"] == r["n_matched"], tag
    for k in ("breaking", "breaking_prev", "arising", "active"):
        assert np.array_equal(ch[k], r[k]), (tag, k)


OPTIONS = [
    dict(),
    dict(events=True, edge_rule=vd.VD_EDGE_VERTEX),
    dict(events=True, match_rule=vd.VD_MATCH_CENTROID, match_radius=6, connectivity=8),
]
ORACLE_OPTS = [
    dict(),
    dict(events=True, edge_rule="vertex"),
    dict(events=True, match="centroid", match_radius=6, connectivity=8),
]


@pytest.mark.parametrize("k", range(len(OPTIONS)))
def test_resumed_context_equals_uninterrupted_run_and_oracle(k):
    Lx, Ly = 230, 170
    frames = list(I.noise_frames(Ly, 2.5, 6, 0.03, seed=40 + k, Lx=Lx))
    dev = [torch.from_numpy(F).cuda() for F in frames]
    ref = O.Detector(Lx, Ly, voronoi="brute", **ORACLE_OPTS[k])
    want = [ref.push(F) for F in frames]
    a = vd.Detector(Lx, Ly, **OPTIONS[k])
    for f in range(3):
        a.push(dev[f])
    blob = a.export_state()
    lab2, cq2, e2 = a.labels(), a.centroids(), a.edges()
    run_a = []
    for f in range(3, 6):
        a.push(dev[f])
        run_a.append(a.changes())
    # a fresh context resumed from the checkpoint
    b = vd.Detector(Lx, Ly, **OPTIONS[k])
    b.import_state(blob)
    K, E, fi = b.counts()
    assert (K, E, fi) == (len(cq2), len(e2), 2)
    assert np.array_equal(b.labels(), lab2) and np.array_equal(b.centroids(), cq2)
    assert np.array_equal(b.edges(), e2)
    for getter in (b.owners, b.changes, b.match):
        with pytest.raises(vd.VdError) as e:
            getter()
        assert e.value.status == vd.VD_ERR_STATE
    for f in range(3, 6):
        b.push(dev[f])
        ch = b.changes()
        assert ch["frame"] == f
        _same_changes(ch, run_a[f - 3], f"resumed frame {f}")
        _oracle_changes_equal(ch, want[f], f"resumed frame {f} vs oracle")
        assert np.array_equal(b.owners(), want[f]["owners"])
    # the same context rolled back to the checkpoint
    a.import_state(blob)
    a.push(dev[3])
    _same_changes(a.changes(), run_a[0], "rolled back")
    a.close()
    b.close()


def test_damaged_or_foreign_blobs_are_refused():
    Lx, Ly = 200, 150
    frames = list(I.noise_frames(Ly, 3.0, 3, 0.02, seed=9, Lx=Lx))
    dev = [torch.from_numpy(F).cuda() for F in frames]
    a = vd.Detector(Lx, Ly)
    a.push(dev[0])
    a.push(dev[1])
    blob = a.export_state()
    b = vd.Detector(Lx, Ly)
    b.push(dev[0])
    rng = np.random.default_rng(3)
    for trial in range(6):
        bad = blob.copy()
        pos = int(rng.integers(0, bad.size))
        bad[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        with pytest.raises(vd.VdError) as e:
            b.import_state(bad)
        assert e.value.status == vd.VD_ERR_INVALID, pos
    with pytest.raises(vd.VdError) as e:
        b.import_state(blob[:-4])
    assert e.value.status == vd.VD_ERR_INVALID
    other = vd.Detector(Lx + 1, Ly)
    with pytest.raises(vd.VdError) as e:
        other.import_state(blob)
    assert e.value.status == vd.VD_ERR_INVALID
    other.close()
    # b is unchanged: its next frame compares against its own frame 0
    b.push(dev[1])
    ref = O.Detector(Lx, Ly)
    ref.push(frames[0])
    _oracle_changes_equal(b.changes(), ref.push(frames[1]), "after refused imports")
    fresh = vd.Detector(Lx, Ly)
    with pytest.raises(vd.VdError) as e:
        fresh.export_state()
    assert e.value.status == vd.VD_ERR_STATE
    for d in (a, b, fresh):
        d.close()


def test_batch_instance_checkpoint_moves_to_a_context_with_walls_and_obstacles():
    """A batch instance (bounded x axis, obstacle posts) exported and resumed
    in a plain context of the same lattice; the obstacle mask is set again."""
    Lx, Ly = 180, 96
    frames = list(I.noise_frames(Ly, 2.5, 4, 0.03, seed=77, Lx=Lx))
    dev = [torch.from_numpy(F).cuda() for F in frames]
    posts = np.zeros((Ly, Lx), bool)
    posts[40:46, 30:36] = True
    posts[60:64, 120:126] = True
    bt = vd.Batch([(128, 128), (Lx, Ly)], options=[{}, dict(walls=vd.VD_WALL_X)])
    bt.set_obstacles(1, posts)
    other = torch.from_numpy(I.smoothed_noise(128, 128, 3.0, seed=1)).cuda()
    for f in range(2):
        bt.push([other, dev[f]])
    blob = bt.export_state(1)
    det = vd.Detector(Lx, Ly, walls=vd.VD_WALL_X)
    det.set_obstacles(posts)
    det.import_state(blob)
    ref = O.Detector(Lx, Ly, walls=(True, False), obstacles=posts)
    for F in frames[:2]:
        ref.push(F)
    for f in (2, 3):
        det.push(dev[f])
        bt.push([other, dev[f]])
        r = ref.push(frames[f])
        _oracle_changes_equal(det.changes(), r, f"walls frame {f}")
        _same_changes(det.changes(), bt.changes(1), f"walls frame {f} vs batch")
        assert np.array_equal(det.labels(), r["labels"])
    det.close()
    bt.close()


def test_c1_checkpoint_mid_sequence():
    """1024^2 smoothed noise (sigma 4): checkpoint after frame 2, resume in a
    fresh context, frames 3-5 equal the oracle."""
    frames = list(I.workload_c1(seed=3, n_frames=6))
    a = vd.Detector(1024, 1024)
    for F in frames[:3]:
        a.push(torch.from_numpy(F).cuda())
    blob = a.export_state()
    a.close()
    b = vd.Detector(1024, 1024)
    b.import_state(blob)
    ref = O.Detector(1024, 1024, workers=-1)
    for F in frames[:3]:
        ref.push(F)
    for f in range(3, 6):
        b.push(torch.from_numpy(frames[f]).cuda())
        r = ref.push(frames[f])
        _oracle_changes_equal(b.changes(), r, f"c1 frame {f}")
        assert np.array_equal(b.edges(), r["edges"])
    b.close()


def test_import_into_a_context_whose_last_frame_overflowed():
    """A context whose last frame overflowed its link list (its link hash
    still holds unlisted keys) imports a checkpoint: the frames after it
    equal the oracle, changes included."""
    L = 128
    dense = I.smoothed_noise(L, L, 1.5, seed=3)
    sparse = list(I.noise_frames(L, 5.0, 3, 0.02, seed=4))
    ref = O.Detector(L, L, voronoi="brute")
    want = [ref.push(F) for F in sparse]
    cap = max(len(r["edges"]) for r in want) + 8
    a = vd.Detector(L, L)
    a.push(torch.from_numpy(sparse[0]).cuda())
    blob = a.export_state()
    a.close()
    b = vd.Detector(L, L, max_edges=cap)
    b.push(torch.from_numpy(dense).cuda())
    with pytest.raises(vd.VdError) as e:
        b.edges()
    assert e.value.status == vd.VD_ERR_CAPACITY
    b.import_state(blob)
    for f in (1, 2):
        b.push(torch.from_numpy(sparse[f]).cuda())
        assert np.array_equal(b.labels(), want[f]["labels"]), f
        assert np.array_equal(b.edges(), want[f]["edges"]), f
        _oracle_changes_equal(b.changes(), want[f], f"frame {f}")
    b.close()
