"""Launch-shape tuning (vd_set_tuning / vd_batch_set_tuning) changes speed only:
every owner-kernel patch layout, bucket scale and first search radius, and
both forms of the graph stage (one block per instance, grid-wide kernels),
give the oracle's labels, owners, links and flips bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402

SETTINGS = [(p, b, r) for p in (vd.VD_PATCH_8x8, vd.VD_PATCH_16x8, vd.VD_PATCH_32x8, vd.VD_PATCH_16x16)
            for b, r in ((100, 9), (40, 0), (250, 40))]


@pytest.fixture(scope="module")
def cases():
    out = []
    for Lx, Ly, sig, seed in ((203, 141, 2.0, 3), (256, 256, 4.0, 5), (96, 300, 1.2, 8)):
        frames = list(I.noise_frames(Ly, sig, 2, 0.03, seed=seed, Lx=Lx))
        ref = O.Detector(Lx, Ly, voronoi="brute")
        out.append((Lx, Ly, frames, [ref.push(F) for F in frames]))
    return out


@pytest.mark.parametrize("patch,bucket_pct,ring0", SETTINGS)
def test_every_tuning_gives_the_oracle_result(cases, patch, bucket_pct, ring0):
    for Lx, Ly, frames, want in cases:
        det = vd.Detector(Lx, Ly)
        det.set_tuning(patch, bucket_pct, ring0)
        t = det.tuning()
        assert (t["voronoi_patch"], t["bucket_pct"], t["ring0"]) == (patch, bucket_pct, ring0)
        for F, r in zip(frames, want):
            det.push(torch.from_numpy(F).cuda())
            tag = (Lx, Ly, patch, bucket_pct, ring0)
            assert np.array_equal(det.owners(), r["owners"]), tag
            assert np.array_equal(det.edges(), r["edges"]), tag
            ch = det.changes()
            assert np.array_equal(ch["breaking"], r["breaking"]) and np.array_equal(ch["arising"], r["arising"]), tag
        det.close()


def test_tuning_is_validated():
    det = vd.Detector(64, 64)
    for bad in ((7, 100, 9), (0, 10, 9), (0, 100, -1), (0, 100, 1000), (0, 100, 9, 2)):
        with pytest.raises(vd.VdError) as e:
            det.set_tuning(*bad)
        assert e.value.status == vd.VD_ERR_INVALID
    det.close()


def test_batch_tuning_changes_nothing_in_the_results():
    """A frame-sequence batch re-captures its graph when the patch layout
    changes between pushes; each push still equals the oracle."""
    Lx = Ly = 192
    frames = list(I.noise_frames(Ly, 2.5, 9, 0.03, seed=31))
    ref = O.Detector(Lx, Ly)
    want = [ref.push(F) for F in frames]
    b = vd.Batch([(Lx, Ly)], sequence=3)
    dev = [torch.from_numpy(F).cuda() for F in frames]
    for k, (patch, bp, r0, gb) in enumerate(((0, 100, 9, 1), (3, 60, 0, 0), (1, 150, 20, 1))):
        b.set_tuning(patch, bp, r0, gb)
        b.push(dev[3 * k: 3 * k + 3])
        for i in range(3):
            r = want[3 * k + i]
            assert np.array_equal(b.owners(i), r["owners"]), (k, i)
            ch = b.changes(i)
            assert np.array_equal(ch["breaking"], r["breaking"]) and np.array_equal(ch["arising"], r["arising"])
    b.close()


@pytest.mark.parametrize("graph_blocks", (0, 1))
@pytest.mark.parametrize("opts", ("plain", "events", "centroid", "vertex"))
def test_graph_stage_forms_give_the_oracle_result(graph_blocks, opts):
    """Both forms of the graph stage, with the options whose work lies in it
    (event classes, the centre match) and the vertex link rule, on a single
    lattice and on a frame sequence (whose instances translate the CSR that
    the previous instance built in the same step)."""
    kw = dict(events=opts == "events", match_rule=vd.VD_MATCH_CENTROID if opts == "centroid" else vd.VD_MATCH_OVERLAP,
              match_radius=3 if opts == "centroid" else 0,
              edge_rule=vd.VD_EDGE_VERTEX if opts == "vertex" else vd.VD_EDGE_ADJ4)
    okw = dict(events=opts == "events", match="centroid" if opts == "centroid" else "overlap",
               match_radius=3 if opts == "centroid" else 0, edge_rule="vertex" if opts == "vertex" else "adj4")
    Lx, Ly = 203, 141
    frames = list(I.noise_frames(Ly, 2.0, 7, 0.03, seed=77, Lx=Lx))
    ref = O.Detector(Lx, Ly, voronoi="brute", **okw)
    want = [ref.push(F) for F in frames]
    dev = [torch.from_numpy(F).cuda() for F in frames]

    def same(ch, r, tag):
        assert np.array_equal(ch["breaking"], r["breaking"]), tag
        assert np.array_equal(ch["breaking_prev"], r["breaking_prev"]), tag
        assert np.array_equal(ch["arising"], r["arising"]), tag
        assert np.array_equal(ch["active"], r["active"]), tag

    det = vd.Detector(Lx, Ly, **kw)
    det.set_tuning(graph_blocks=graph_blocks)
    assert det.tuning()["graph_blocks"] == graph_blocks
    for f, (F, r) in enumerate(zip(dev, want)):
        det.push(F)
        assert np.array_equal(det.edges(), r["edges"]), f
        same(det.changes(), r, ("single", f))
        if r["K_prev"]:
            assert np.array_equal(det.match(), r["phi"]), f
    det.close()
    b = vd.Batch([(Lx, Ly)], sequence=3, **kw)
    b.set_tuning(graph_blocks=graph_blocks)
    b.push(dev[0:3])
    b.push(dev[3:6])
    for i in range(3):
        same(b.changes(i), want[3 + i], ("sequence", 3 + i))
    b.close()
