"""The one device-side wait of a step gives up instead of hanging.

The prefix scans of a step use a decoupled look-back: a scan tile waits for
its predecessors' flags. Every such wait is bounded; when it runs out the
frame reports VD_ERR_TIMEOUT and the context stays usable. The test makes a
wait run out on purpose: a test hook (vd_debug_hold_scan_flag) makes one scan
tile withhold its flag -- a flag that nothing sets -- so its successor polls a
bounded number of times and returns. Nothing here faults, traps or hangs the
GPU: the withheld flag only changes which branch of the bounded loop runs.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402

RANK_SCAN = 0   # the bubble-rank scan: 2048^2 has 2048 x 8 root groups = 4 scan tiles


def _check_against_oracle(det, r, tag):
    K, E, _ = det.counts()
    assert K == r["K"], tag
    assert np.array_equal(det.labels(), r["labels"]), tag
    assert np.array_equal(det.centroids(), r["centroids"]), tag
    assert np.array_equal(det.owners(), r["owners"]), tag
    assert np.array_equal(det.edges(), r["edges"]), tag
    ch = det.changes()
    for k in ("breaking", "breaking_prev", "arising", "active"):
        assert np.array_equal(ch[k], r[k]), (tag, k)


@pytest.mark.parametrize("spin_limit", [64, 0])
def test_scan_wait_gives_up_with_timeout_and_context_recovers(spin_limit):
    L = 2048
    frames = list(I.noise_frames(L, 4.0, 4, 0.005, seed=21))
    dev = [torch.from_numpy(F).cuda() for F in frames]
    det = vd.Detector(L, L)
    det.push(dev[0])
    det.counts()
    # tile 1 withholds its flag: tile 2's look-back finds it never ready
    det.hold_scan_flag(RANK_SCAN, 1, spin_limit)
    t0 = time.perf_counter()
    det.push(dev[1])
    with pytest.raises(vd.VdError) as e:
        det.changes()
    elapsed = time.perf_counter() - t0
    assert e.value.status == vd.VD_ERR_TIMEOUT
    with pytest.raises(vd.VdError) as e:
        det.labels()
    assert e.value.status == vd.VD_ERR_TIMEOUT
    # the default limit (2^20 polls) is about a second; the short one much less
    assert elapsed < (2.0 if spin_limit else 30.0), elapsed
    det.hold_scan_flag(RANK_SCAN, -1)
    # a frame after the failed one has no past frame; the one after it is a
    # regular pair -- both equal the oracle run on those two frames alone
    ref = O.Detector(L, L, workers=-1)
    det.push(dev[2])
    _check_against_oracle(det, ref.push(frames[2]), "frame after the timeout")
    det.push(dev[3])
    _check_against_oracle(det, ref.push(frames[3]), "next frame")
    det.close()
