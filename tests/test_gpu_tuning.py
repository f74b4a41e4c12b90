"""Launch-shape tuning (vd_set_tuning / vd_batch_set_tuning) changes speed only:
every owner-kernel patch layout, bucket scale and first search radius gives
the oracle's labels, owners, links and flips bit for bit."""
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
        assert det.tuning() == dict(voronoi_patch=patch, bucket_pct=bucket_pct, ring0=ring0)
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
    for bad in ((7, 100, 9), (0, 10, 9), (0, 100, -1), (0, 100, 1000)):
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
    for k, (patch, bp, r0) in enumerate(((0, 100, 9), (3, 60, 0), (1, 150, 20))):
        b.set_tuning(patch, bp, r0)
        b.push(dev[3 * k: 3 * k + 3])
        for i in range(3):
            r = want[3 * k + i]
            assert np.array_equal(b.owners(i), r["owners"]), (k, i)
            ch = b.changes(i)
            assert np.array_equal(ch["breaking"], r["breaking"]) and np.array_equal(ch["arising"], r["arising"])
    b.close()
