"""The checked build (libvd_checked.so: the same kernels compiled with
-DVD_CHECKED, an index test before every data-dependent scatter access).

It stands in for a memory checker: the parity tests run again with the
checked library loaded (VD_LIB=checked, in a child process, since a process
loads one libvd), where any failed index test would make the getters return
VD_ERR_BOUNDS and fail the comparison; and the reporting path is exercised by
the test hook that makes one check fail without any access (the flip-list
check, whose skipped writes feed no later index).
"""
from __future__ import annotations

import os
import re
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.environ.get("VD_LIB") == "checked"
CHK_FLIPS = 18

SUBSET = " or ".join((
    "test_c0_two_frames", "test_random_small_lattices", "test_degenerate_fields", "test_wide_bubbles_across_seams",
    "test_tiny_lattices", "test_pitched_field", "test_c1_frames", "test_capacity_overflow_is_reported",
    "test_event_classes_with_boundary_points", "test_centroid_match_sequences", "test_eight_connectivity",
    "test_vertex_link_rule", "test_walls_and_obstacles", "test_uneven_batch_matches_per_instance_oracle",
    "test_batch_with_mixed_options", "test_frame_sequence_matches_oracle", "overflow_then_exact_frames",
    "test_many_instances_and_a_long_sequence", "test_every_tuning_gives_the_oracle_result",
    "test_graph_stage_forms_give_the_oracle_result", "test_resumed_context_equals_uninterrupted_run_and_oracle",
    "test_import_into_a_context_whose_last_frame_overflowed", "test_pieces_per_tile_at_the_shared_sum_limit",
))


def _child(args, timeout):
    env = dict(os.environ, VD_LIB="checked", VD_FULL="0")
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


@pytest.mark.skipif(CHECKED, reason="already running under the checked build")
def test_parity_suite_under_the_checked_build():
    r = _child(["-m", "pytest", "tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "tests/test_gpu_tuning.py",
                "tests/test_gpu_state.py", "tests/test_gpu_checked.py", "-m", "gpu", "-q", "-x", "-p",
                "no:cacheprovider", "-k", SUBSET + " or test_loaded_library"], 1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 60 and " failed" not in r.stdout, tail


def test_loaded_library():
    """The regular build reports itself unchecked; the checked one checked."""
    det = vd.Detector(64, 48)
    det.push(torch.zeros((48, 64), dtype=torch.float32, device="cuda"))
    info = det.check_info()
    assert info["checked"] is CHECKED
    assert info["first_check"] == 0
    det.close()


@pytest.mark.skipif(CHECKED, reason="runs its own child process")
def test_checked_build_reports_a_failed_check():
    r = _child(["-c", "import tests.test_gpu_checked as t; t.forced_check_run()"], 600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    assert "forced check ok" in r.stdout, r.stdout[-2000:]


def forced_check_run():
    """Body of the reporting test (child process, checked library)."""
    assert vd.LIB_PATH.endswith("libvd_checked.so")
    L = 192
    frames = list(I.noise_frames(L, 3.0, 4, 0.02, seed=21))
    det = vd.Detector(L, L)
    ref = O.Detector(L, L, workers=-1)
    dev = [torch.from_numpy(np.ascontiguousarray(F)).cuda() for F in frames]
    det.push(dev[0])
    ref.push(frames[0])
    assert det.check_info() == dict(checked=True, first_check=0, index=0)
    # frame 1 with the flip-list check forced to fail: the flips are not
    # written, every getter of the frame reports VD_ERR_BOUNDS
    det.force_check(CHK_FLIPS)
    det.push(dev[1])
    r1 = ref.push(frames[1])
    assert len(r1["breaking"]) + len(r1["arising"]) > 0, "the frame must have flips"
    with pytest.raises(vd.VdError) as e:
        det.changes()
    assert e.value.status == vd.VD_ERR_BOUNDS
    info = det.check_info()
    assert info["checked"] and info["first_check"] == CHK_FLIPS and info["index"] >= 0
    # hook off: the next frame is exact but has no past frame (a failed frame
    # is never used as one); the frame after it is exact in every output
    det.force_check(0)
    det.push(dev[2])
    r2 = ref.push(frames[2])
    assert det.check_info()["first_check"] == 0
    assert np.array_equal(det.labels(), r2["labels"]) and np.array_equal(det.owners(), r2["owners"])
    assert np.array_equal(det.edges(), r2["edges"])
    assert det.changes()["K_prev"] == 0
    det.push(dev[3])
    r3 = ref.push(frames[3])
    ch = det.changes()
    assert np.array_equal(det.labels(), r3["labels"]) and np.array_equal(det.edges(), r3["edges"])
    assert np.array_equal(ch["breaking"], r3["breaking"]) and np.array_equal(ch["arising"], r3["arising"])
    assert np.array_equal(ch["active"], r3["active"])
    det.close()
    print("forced check ok")
