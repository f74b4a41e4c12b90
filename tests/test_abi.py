"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol that include/vd.h declares, and argument validation needs no GPU."""
import os
import re

import pytest

from paper_1607_00908_gb300 import vd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(vd.LIB_PATH):
        from paper_1607_00908_gb300 import build
        build.build()
    return vd.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "vd.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vd_status|const char\*)\s+(vd_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi():
    names = declared_symbols()
    assert "vd_create" in names and "vd_push_frame" in names and "vd_get_changes" in names
    assert "vd_destroy" in names and "vd_batch_push" in names
    assert sorted(vd.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert vd.status_string(vd.VD_OK) == "ok"
    assert vd.status_string(vd.VD_ERR_CAPACITY) == "capacity exceeded"
    assert vd.status_string(12345) == "unknown status"


@pytest.mark.parametrize("field,value", [("Lx", 0), ("Ly", -3), ("connectivity", 6), ("polarity", 0),
                                         ("Lx", 1 << 21), ("max_components", -1), ("events", 2),
                                         ("match_rule", 7), ("match_radius", -1), ("edge_rule", 3),
                                         ("walls", 4), ("walls", -1), ("max_edges", -1), ("polarity", 2)])
def test_invalid_config_is_rejected_without_touching_the_gpu(lib, field, value):
    cfg = vd.vd_config_init(16, 16)
    setattr(cfg, field, value)
    import ctypes as C
    h = C.c_void_p()
    assert lib.vd_create(C.byref(cfg), C.byref(h)) == vd.VD_ERR_INVALID
    assert lib.vd_batch_create(C.byref(cfg), 1, C.byref(h)) == vd.VD_ERR_INVALID
    assert lib.vd_batch_create(C.byref(cfg), 0, C.byref(h)) == vd.VD_ERR_INVALID


def test_null_handles_are_rejected(lib):
    import ctypes as C
    assert lib.vd_push_frame(None, None, 16) == vd.VD_ERR_INVALID
    assert lib.vd_get_changes(None, None) == vd.VD_ERR_INVALID
    assert lib.vd_destroy(None) == vd.VD_ERR_INVALID
    assert lib.vd_batch_destroy(None) == vd.VD_ERR_INVALID
    assert lib.vd_config_init(None, 4, 4) == vd.VD_ERR_INVALID


def test_centre_match_needs_a_radius_and_walls_double_the_limit(lib):
    """VD_MATCH_CENTROID without a radius is refused; a bounded axis runs with
    twice its length, so its length limit is half that of a periodic axis."""
    import ctypes as C
    h = C.c_void_p()
    cfg = vd.vd_config_init(16, 16, match_rule=vd.VD_MATCH_CENTROID, match_radius=0)
    assert lib.vd_create(C.byref(cfg), C.byref(h)) == vd.VD_ERR_INVALID
    cfg = vd.vd_config_init((1 << 20) + 1, 1, walls=vd.VD_WALL_X)
    assert lib.vd_create(C.byref(cfg), C.byref(h)) == vd.VD_ERR_INVALID
    cfg = vd.vd_config_init(16, 16, match_rule=vd.VD_MATCH_CENTROID, match_radius=(1 << 20) + 1)
    assert lib.vd_create(C.byref(cfg), C.byref(h)) == vd.VD_ERR_INVALID
    # each axis within its limit, but Lx * Ly sites would not fit a 32-bit site index
    cfg = vd.vd_config_init(50000, 50000)
    assert lib.vd_create(C.byref(cfg), C.byref(h)) == vd.VD_ERR_INVALID
    cfg = vd.vd_config_init((1 << 20) + 1, 1)
    st = lib.vd_create(C.byref(cfg), C.byref(h))
    assert st != vd.VD_ERR_INVALID   # a valid config (without a GPU it fails later, at allocation)
    if st == vd.VD_OK:
        lib.vd_destroy(h)
