"""ctypes binding of libvd (include/vd.h): argument marshalling only.

Every function of the C ABI is exposed under the same name. ``Detector`` and
``Batch`` are small conveniences that own a context, take torch CUDA tensors
(device memory and the current stream come from PyTorch) and return numpy
arrays from the getters. All computation happens in libvd's CUDA kernels;
there is no fallback: if libvd.so is missing or cannot be loaded, every call
raises ``VdUnavailable``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VD_LIB=checked selects the checked build (index checks, include/vd.h)
LIB_PATH = os.path.join(_HERE, "libvd_checked.so" if os.environ.get("VD_LIB") == "checked" else "libvd.so")

VD_OK = 0
VD_ERR_INVALID = -1
VD_ERR_OOM = -2
VD_ERR_CAPACITY = -3
VD_ERR_CUDA = -4
VD_ERR_TIMEOUT = -5
VD_ERR_STATE = -6
VD_ERR_UNSUPPORTED = -7
VD_ERR_BOUNDS = -8
VD_ABOVE = 1
VD_BELOW = -1
# per-label flags of the `active` arrays (bit 0: local trigger; event classes above it)
VD_EV_ACTIVE, VD_EV_BULK, VD_EV_BOUNDARY, VD_EV_BPOINT_NOW, VD_EV_BPOINT_PAST = 1, 2, 4, 8, 16
# isomorphism rules (Section 3.2.3)
VD_MATCH_OVERLAP, VD_MATCH_CENTROID = 0, 1
# link rules (Section 3.2.2)
VD_EDGE_ADJ4, VD_EDGE_VERTEX = 0, 1
# bounded axes and the owner of obstacle sites
VD_WALL_X, VD_WALL_Y = 1, 2
VD_OWNER_OBSTACLE = -2

#: every symbol include/vd.h declares
EXPORTS = (
    "vd_config_init", "vd_set_obstacles", "vd_batch_set_obstacles", "vd_create", "vd_push_frame",
    "vd_push_frame_host", "vd_get_changes",
    "vd_get_counts", "vd_get_labels", "vd_get_centroids_q10", "vd_get_owners", "vd_get_edges",
    "vd_get_match", "vd_export_state", "vd_import_state", "vd_set_tuning", "vd_get_tuning",
    "vd_debug_hold_scan_flag", "vd_debug_check_info", "vd_debug_force_check",
    "vd_batch_debug_check_info", "vd_batch_debug_force_check", "vd_set_timing", "vd_get_timing", "vd_stage_name", "vd_destroy", "vd_status_string",
    "vd_batch_create", "vd_batch_create_sequence", "vd_batch_push", "vd_batch_push_host", "vd_batch_push_subset", "vd_batch_get_changes",
    "vd_batch_stage_host", "vd_batch_push_staged", "vd_batch_get_changes_all",
    "vd_batch_get_labels", "vd_batch_get_owners", "vd_batch_get_edges", "vd_batch_get_centroids_q10",
    "vd_batch_get_counts", "vd_batch_set_timing", "vd_batch_get_timing", "vd_batch_destroy",
    "vd_batch_export_state", "vd_batch_import_state", "vd_batch_set_tuning", "vd_batch_get_tuning",
    "vd_voronoi_owners_static", "vd_server_create", "vd_server_open_sim", "vd_server_close_sim",
    "vd_server_clock_ns", "vd_server_submit", "vd_server_poll", "vd_server_keep_changes",
    "vd_server_get_frame_changes", "vd_server_get_changes", "vd_server_get_labels", "vd_server_export_state",
    "vd_server_import_state", "vd_server_stats", "vd_server_destroy",
)


class VdUnavailable(RuntimeError):
    pass


class VdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class vd_config(C.Structure):
    _fields_ = [
        ("Lx", C.c_int32), ("Ly", C.c_int32), ("threshold", C.c_float), ("polarity", C.c_int32),
        ("connectivity", C.c_int32), ("max_components", C.c_int32), ("max_edges", C.c_int32),
        ("stream", C.c_void_p), ("events", C.c_int32), ("match_rule", C.c_int32), ("match_radius", C.c_int32),
        ("edge_rule", C.c_int32), ("walls", C.c_int32),
    ]


class vd_changes(C.Structure):
    _fields_ = [
        ("frame_index", C.c_int64), ("n_prev", C.c_int32), ("n_now", C.c_int32),
        ("n_matched", C.c_int32), ("n_edges", C.c_int32), ("n_breaking", C.c_int32),
        ("n_arising", C.c_int32), ("global_trigger", C.c_int32),
        ("breaking", C.POINTER(C.c_uint64)), ("cap_breaking", C.c_int32),
        ("breaking_prev", C.POINTER(C.c_uint64)),
        ("arising", C.POINTER(C.c_uint64)), ("cap_arising", C.c_int32),
        ("active", C.POINTER(C.c_uint8)), ("cap_active", C.c_int32),
    ]


class vd_tuning(C.Structure):
    _fields_ = [("voronoi_patch", C.c_int32), ("bucket_pct", C.c_int32), ("ring0", C.c_int32),
                ("graph_blocks", C.c_int32)]


VD_PATCH_8x8, VD_PATCH_16x8, VD_PATCH_32x8, VD_PATCH_16x16 = 0, 1, 2, 3


class vd_batch_changes(C.Structure):
    _fields_ = [
        ("status", C.POINTER(C.c_int32)), ("n_prev", C.POINTER(C.c_int32)), ("n_now", C.POINTER(C.c_int32)),
        ("n_breaking", C.POINTER(C.c_int32)), ("n_arising", C.POINTER(C.c_int32)),
        ("breaking", C.POINTER(C.c_uint64)), ("breaking_prev", C.POINTER(C.c_uint64)), ("cap_breaking", C.c_int64),
        ("arising", C.POINTER(C.c_uint64)), ("cap_arising", C.c_int64),
        ("active", C.POINTER(C.c_uint8)), ("cap_active", C.c_int64),
        ("total_breaking", C.c_int64), ("total_arising", C.c_int64), ("total_active", C.c_int64),
    ]


class vd_server_done(C.Structure):
    _fields_ = [
        ("ticket", C.c_int64), ("sim", C.c_int32), ("status", C.c_int32),
        ("t_arrival_ns", C.c_int64), ("t_submit_ns", C.c_int64), ("t_done_ns", C.c_int64),
        ("n_bubbles", C.c_int32), ("n_edges", C.c_int32), ("n_breaking", C.c_int32), ("n_arising", C.c_int32),
    ]


_lib = None


def lib():
    """Load libvd.so (built by ``paper_1607_00908_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise VdUnavailable(f"{LIB_PATH} is missing: run paper_1607_00908_gb300.build.build() first")
    try:
        L = C.CDLL(LIB_PATH)
    except OSError as e:
        raise VdUnavailable(f"cannot load {LIB_PATH}: {e}") from e
    P, I32, I64, VP = C.POINTER, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "vd_config_init": [P(vd_config), I32, I32],
        "vd_set_obstacles": [C.c_void_p, C.c_void_p, C.c_int64],
        "vd_batch_set_obstacles": [C.c_void_p, I32, C.c_void_p, C.c_int64],
        "vd_create": [P(vd_config), P(VP)],
        "vd_push_frame": [VP, VP, C.c_size_t],
        "vd_push_frame_host": [VP, VP, C.c_size_t],
        "vd_get_changes": [VP, P(vd_changes)],
        "vd_get_counts": [VP, P(I32), P(I32), P(I64)],
        "vd_get_labels": [VP, VP, I64, P(I64)],
        "vd_get_centroids_q10": [VP, VP, I64, P(I64)],
        "vd_get_owners": [VP, VP, I64, P(I64)],
        "vd_get_edges": [VP, VP, I64, P(I64)],
        "vd_get_match": [VP, VP, I64, P(I64)],
        "vd_export_state": [VP, VP, I64, P(I64)],
        "vd_import_state": [VP, VP, I64],
        "vd_batch_export_state": [VP, I32, VP, I64, P(I64)],
        "vd_batch_import_state": [VP, I32, VP, I64],
        "vd_debug_hold_scan_flag": [VP, I32, I64, I32],
        "vd_debug_check_info": [VP, P(I32), P(I32), P(I64)],
        "vd_debug_force_check": [VP, I32],
        "vd_batch_debug_check_info": [VP, P(I32), P(I32), P(I64)],
        "vd_batch_debug_force_check": [VP, I32],
        "vd_set_tuning": [VP, P(vd_tuning)],
        "vd_get_tuning": [VP, P(vd_tuning)],
        "vd_batch_set_tuning": [VP, P(vd_tuning)],
        "vd_batch_get_tuning": [VP, P(vd_tuning)],
        "vd_set_timing": [VP, I32],
        "vd_get_timing": [VP, P(C.c_double), I32, P(I32), P(I64), P(I64)],
        "vd_stage_name": [I32],
        "vd_destroy": [VP],
        "vd_status_string": [I32],
        "vd_batch_create": [P(vd_config), I32, P(VP)],
        "vd_batch_create_sequence": [P(vd_config), I32, P(VP)],
        "vd_batch_push": [VP, P(VP)],
        "vd_batch_push_host": [VP, P(VP)],
        "vd_batch_push_subset": [VP, P(I32), I32, P(VP)],
        "vd_batch_get_changes": [VP, I32, P(vd_changes)],
        "vd_batch_stage_host": [VP, P(VP)],
        "vd_batch_push_staged": [VP],
        "vd_batch_get_changes_all": [VP, P(vd_batch_changes)],
        "vd_batch_get_labels": [VP, I32, VP, I64, P(I64)],
        "vd_batch_get_owners": [VP, I32, VP, I64, P(I64)],
        "vd_batch_get_edges": [VP, I32, VP, I64, P(I64)],
        "vd_batch_get_centroids_q10": [VP, I32, VP, I64, P(I64)],
        "vd_batch_get_counts": [VP, I32, P(I32), P(I32), P(I64)],
        "vd_batch_set_timing": [VP, I32],
        "vd_batch_get_timing": [VP, P(C.c_double), I32, P(I32), P(I64), P(I64)],
        "vd_batch_destroy": [VP],
        "vd_voronoi_owners_static": [VP, I32, I32, I32, VP, VP],
        "vd_server_create": [P(vd_config), I32, I64, I32, VP, P(VP)],
        "vd_server_open_sim": [VP, P(vd_config), P(I32)],
        "vd_server_close_sim": [VP, I32],
        "vd_server_clock_ns": [P(I64)],
        "vd_server_submit": [VP, I32, VP, I64, P(I64)],
        "vd_server_poll": [VP, I32, P(vd_server_done), I32, P(I32)],
        "vd_server_keep_changes": [VP, I32],
        "vd_server_get_frame_changes": [VP, I64, P(vd_changes)],
        "vd_server_get_changes": [VP, I32, P(vd_changes)],
        "vd_server_get_labels": [VP, I32, VP, I64, P(I64)],
        "vd_server_export_state": [VP, I32, VP, I64, P(I64)],
        "vd_server_import_state": [VP, I32, VP, I64],
        "vd_server_stats": [VP, P(I64), P(I64), P(I64), P(I64)],
        "vd_server_destroy": [VP],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_char_p if name in ("vd_status_string", "vd_stage_name") else C.c_int32
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().vd_status_string(int(s)).decode()


def _check(s: int, where: str):
    if s != VD_OK:
        raise VdError(s, where)


# ----------------------------------------------------------------------------
# raw C-ABI names
# ----------------------------------------------------------------------------

def vd_config_init(Lx: int, Ly: int, threshold: float = 0.5, polarity: int = VD_ABOVE,
                   stream: int | None = None, max_components: int = 0, max_edges: int = 0,
                   events: bool = False, match_rule: int = VD_MATCH_OVERLAP, match_radius: int = 0,
                   connectivity: int = 4, edge_rule: int = VD_EDGE_ADJ4, walls: int = 0) -> vd_config:
    cfg = vd_config()
    _check(lib().vd_config_init(C.byref(cfg), int(Lx), int(Ly)), "vd_config_init")
    cfg.threshold = float(threshold)
    cfg.polarity = int(polarity)
    cfg.max_components = int(max_components)
    cfg.max_edges = int(max_edges)
    cfg.stream = C.c_void_p(stream or 0)
    cfg.events = int(bool(events))
    cfg.match_rule = int(match_rule)
    cfg.match_radius = int(match_radius)
    cfg.connectivity = int(connectivity)
    cfg.edge_rule = int(edge_rule)
    cfg.walls = int(walls)
    return cfg


def vd_create(cfg: vd_config) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().vd_create(C.byref(cfg), C.byref(h)), "vd_create")
    return h


def vd_push_frame(ctx, d_field_ptr: int, pitch: int) -> int:
    return lib().vd_push_frame(ctx, C.c_void_p(d_field_ptr), pitch)


def vd_push_frame_host(ctx, h_field_ptr: int, pitch: int) -> int:
    return lib().vd_push_frame_host(ctx, C.c_void_p(h_field_ptr), pitch)


def vd_get_changes(ctx, out: vd_changes) -> int:
    return lib().vd_get_changes(ctx, C.byref(out))


def vd_get_counts(ctx):
    K, E, f = C.c_int32(), C.c_int32(), C.c_int64()
    s = lib().vd_get_counts(ctx, C.byref(K), C.byref(E), C.byref(f))
    return s, K.value, E.value, f.value


def vd_get_labels(ctx, out_ptr: int, cap: int):
    n = C.c_int64()
    return lib().vd_get_labels(ctx, C.c_void_p(out_ptr), cap, C.byref(n)), n.value


def vd_get_owners(ctx, out_ptr: int, cap: int):
    n = C.c_int64()
    return lib().vd_get_owners(ctx, C.c_void_p(out_ptr), cap, C.byref(n)), n.value


def vd_get_centroids_q10(ctx, out_ptr: int, cap: int):
    n = C.c_int64()
    return lib().vd_get_centroids_q10(ctx, C.c_void_p(out_ptr), cap, C.byref(n)), n.value


def vd_get_edges(ctx, out_ptr: int, cap: int):
    n = C.c_int64()
    return lib().vd_get_edges(ctx, C.c_void_p(out_ptr), cap, C.byref(n)), n.value


def vd_get_match(ctx, out_ptr: int, cap: int):
    n = C.c_int64()
    return lib().vd_get_match(ctx, C.c_void_p(out_ptr), cap, C.byref(n)), n.value


def vd_destroy(ctx) -> int:
    return lib().vd_destroy(ctx)


def vd_batch_create(cfgs) -> C.c_void_p:
    arr = (vd_config * len(cfgs))(*cfgs)
    h = C.c_void_p()
    _check(lib().vd_batch_create(arr, len(cfgs), C.byref(h)), "vd_batch_create")
    return h


def vd_batch_push(b, field_ptrs) -> int:
    arr = (C.c_void_p * len(field_ptrs))(*[C.c_void_p(p) for p in field_ptrs])
    return lib().vd_batch_push(b, arr)


def vd_batch_push_subset(b, active, field_ptrs) -> int:
    act = (C.c_int32 * len(active))(*active)
    arr = (C.c_void_p * len(field_ptrs))(*[C.c_void_p(p) for p in field_ptrs])
    return lib().vd_batch_push_subset(b, act, len(active), arr)


def vd_batch_get_changes(b, i: int, out: vd_changes) -> int:
    return lib().vd_batch_get_changes(b, i, C.byref(out))


def vd_batch_get_counts(b, i: int):
    K, E, f = C.c_int32(), C.c_int32(), C.c_int64()
    s = lib().vd_batch_get_counts(b, i, C.byref(K), C.byref(E), C.byref(f))
    return s, K.value, E.value, f.value


def vd_batch_destroy(b) -> int:
    return lib().vd_batch_destroy(b)


def vd_voronoi_owners_static(d_centroids_ptr: int, K: int, Lx: int, Ly: int, d_owners_ptr: int,
                             stream: int = 0) -> int:
    return lib().vd_voronoi_owners_static(C.c_void_p(d_centroids_ptr), K, Lx, Ly, C.c_void_p(d_owners_ptr),
                                          C.c_void_p(stream))


# ----------------------------------------------------------------------------
# conveniences
# ----------------------------------------------------------------------------

def _changes(getter, K_now: int, cap: int):
    brk = np.empty(max(cap, 1), np.uint64)
    brkp = np.empty(max(cap, 1), np.uint64)
    ari = np.empty(max(cap, 1), np.uint64)
    act = np.empty(max(K_now, 1), np.uint8)
    ch = vd_changes()
    ch.breaking = brk.ctypes.data_as(C.POINTER(C.c_uint64))
    ch.breaking_prev = brkp.ctypes.data_as(C.POINTER(C.c_uint64))
    ch.arising = ari.ctypes.data_as(C.POINTER(C.c_uint64))
    ch.active = act.ctypes.data_as(C.POINTER(C.c_uint8))
    ch.cap_breaking = cap
    ch.cap_arising = cap
    ch.cap_active = max(K_now, 1)
    s = getter(ch)
    return s, ch, brk, brkp, ari, act


class _Base:
    _get_counts = None

    def _read(self, getter_name, i, dtype, count, mult=1):
        out = np.empty(max(count * mult, 1), dtype=dtype)
        n = C.c_int64()
        fn = getattr(lib(), getter_name)
        args = (self.h,) if i is None else (self.h, i)
        s = fn(*args, out.ctypes.data_as(C.c_void_p), out.size, C.byref(n))
        _check(s, getter_name)
        return out[: n.value]


class Detector(_Base):
    """One periodic lattice (vd_create / vd_push_frame / vd_get_* / vd_destroy)."""

    def __init__(self, Lx: int, Ly: int, threshold: float = 0.5, polarity: int = VD_ABOVE,
                 stream: int | None = None, max_components: int = 0, max_edges: int = 0,
                 events: bool = False, match_rule: int = VD_MATCH_OVERLAP, match_radius: int = 0,
                 connectivity: int = 4, edge_rule: int = VD_EDGE_ADJ4, walls: int = 0):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.Lx, self.Ly = Lx, Ly
        self.cfg = vd_config_init(Lx, Ly, threshold, polarity, stream, max_components, max_edges,
                                  events, match_rule, match_radius, connectivity, edge_rule, walls)
        self.h = vd_create(self.cfg)

    def set_obstacles(self, mask) -> None:
        """mask: host array [Ly, Lx], nonzero = obstacle site (vd_set_obstacles)."""
        import numpy as np
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        _check(lib().vd_set_obstacles(self.h, m.ctypes.data, m.shape[1]), "vd_set_obstacles")

    def push(self, field) -> None:
        """field: torch CUDA float32 tensor [Ly, Lx] (row stride = field.stride(0))."""
        assert field.is_cuda and field.dtype.itemsize == 4 and field.stride(1) == 1
        _check(vd_push_frame(self.h, field.data_ptr(), field.stride(0)), "vd_push_frame")

    def push_host(self, arr: np.ndarray) -> None:
        a = np.ascontiguousarray(arr, dtype=np.float32)
        _check(vd_push_frame_host(self.h, a.ctypes.data, a.shape[1]), "vd_push_frame_host")

    def counts(self):
        s, K, E, f = vd_get_counts(self.h)
        _check(s, "vd_get_counts")
        return K, E, f

    def labels(self) -> np.ndarray:
        return self._read("vd_get_labels", None, np.int32, self.Lx * self.Ly).reshape(self.Ly, self.Lx)

    def owners(self) -> np.ndarray:
        return self._read("vd_get_owners", None, np.int32, self.Lx * self.Ly).reshape(self.Ly, self.Lx)

    def centroids(self) -> np.ndarray:
        K, _, _ = self.counts()
        return self._read("vd_get_centroids_q10", None, np.int32, K, 2).reshape(-1, 2)

    def edges(self) -> np.ndarray:
        _, E, _ = self.counts()
        return self._read("vd_get_edges", None, np.uint64, E)

    def match(self) -> np.ndarray:
        """Phi: past label -> now label (-1 unmatched), one entry per past bubble."""
        return self._read("vd_get_match", None, np.int32, self.changes()["K_prev"])

    def changes(self) -> dict:
        K, E, _ = self.counts()
        cap = max(E, 1) * 2 + 16
        s, ch, brk, brkp, ari, act = _changes(lambda c: vd_get_changes(self.h, c), K, cap)
        _check(s, "vd_get_changes")
        return dict(frame=ch.frame_index, K_prev=ch.n_prev, K=ch.n_now, n_matched=ch.n_matched,
                    n_edges=ch.n_edges, breaking=brk[: ch.n_breaking].copy(),
                    breaking_prev=brkp[: ch.n_breaking].copy(), arising=ari[: ch.n_arising].copy(),
                    active=act[: ch.n_now].copy(), global_trigger=ch.global_trigger)

    def set_tuning(self, voronoi_patch: int = 0, bucket_pct: int = 100, ring0: int = 9,
                   graph_blocks: int | None = None) -> None:
        """Launch shapes (vd_set_tuning); results are identical for every setting.
        graph_blocks None keeps the current graph-stage form."""
        gb = self.tuning()["graph_blocks"] if graph_blocks is None else int(graph_blocks)
        t = vd_tuning(int(voronoi_patch), int(bucket_pct), int(ring0), gb)
        _check(lib().vd_set_tuning(self.h, C.byref(t)), "vd_set_tuning")

    def tuning(self) -> dict:
        t = vd_tuning()
        _check(lib().vd_get_tuning(self.h, C.byref(t)), "vd_get_tuning")
        return dict(voronoi_patch=t.voronoi_patch, bucket_pct=t.bucket_pct, ring0=t.ring0,
                    graph_blocks=t.graph_blocks)

    def export_state(self) -> np.ndarray:
        """Checkpoint of the last frame's state (vd_export_state), as bytes."""
        n = C.c_int64()
        s = lib().vd_export_state(self.h, None, 0, C.byref(n))
        if s != VD_ERR_CAPACITY:
            _check(s, "vd_export_state")
        buf = np.empty(n.value, np.uint8)
        _check(lib().vd_export_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.size, C.byref(n)), "vd_export_state")
        return buf

    def import_state(self, blob) -> None:
        """Resume from a checkpoint (vd_import_state)."""
        b = np.ascontiguousarray(np.frombuffer(bytes(blob), np.uint8) if not isinstance(blob, np.ndarray) else blob,
                                 dtype=np.uint8)
        _check(lib().vd_import_state(self.h, b.ctypes.data_as(C.c_void_p), b.size), "vd_import_state")

    def hold_scan_flag(self, kind: int, tile: int, spin_limit: int = 0) -> None:
        """Test support: scan tile `tile` of scan `kind` withholds its look-back
        flag in the following pushes (tile -1: off), so the next tile's
        bounded wait runs out (vd_debug_hold_scan_flag)."""
        _check(lib().vd_debug_hold_scan_flag(self.h, int(kind), int(tile), int(spin_limit)),
               "vd_debug_hold_scan_flag")

    def check_info(self) -> dict:
        """Checked build: whether this library checks indices, and the first
        failed check of the last push (id 0: none) with its index."""
        c, i, x = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().vd_debug_check_info(self.h, C.byref(c), C.byref(i), C.byref(x)), "vd_debug_check_info")
        return dict(checked=bool(c.value), first_check=i.value, index=x.value)

    def force_check(self, check_id: int) -> None:
        """Test support: check `check_id` fails from the next push on (0: off)."""
        _check(lib().vd_debug_force_check(self.h, int(check_id)), "vd_debug_force_check")

    def set_timing(self, on: bool) -> None:
        _check(lib().vd_set_timing(self.h, int(bool(on))), "vd_set_timing")

    def timing(self):
        """(per-stage ms since the last call, stage names, kernel launches, frames)."""
        ms = (C.c_double * 16)()
        n, kl, nf = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().vd_get_timing(self.h, ms, 16, C.byref(n), C.byref(kl), C.byref(nf)), "vd_get_timing")
        names = [lib().vd_stage_name(i).decode() for i in range(n.value)]
        return list(ms[: n.value]), names, kl.value, nf.value

    def close(self):
        if getattr(self, "h", None):
            vd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(_Base):
    """Many lattices advanced together (vd_batch_*); with ``sequence=n`` one
    lattice whose push takes n consecutive frames (vd_batch_create_sequence)."""

    def __init__(self, sizes, threshold: float = 0.5, polarity: int = VD_ABOVE, stream: int | None = None,
                 max_components: int = 0, sequence: int = 0, events: bool = False,
                 match_rule: int = VD_MATCH_OVERLAP, match_radius: int = 0, connectivity: int = 4,
                 edge_rule: int = VD_EDGE_ADJ4, walls: int = 0, options=None):
        """``options``: optional list of per-instance dicts of config options
        (events, match_rule, match_radius, connectivity, edge_rule, walls) for
        an independent batch; they replace the keyword defaults instance by
        instance."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.sizes = [(int(lx), int(ly)) for lx, ly in sizes]
        opts = dict(events=events, match_rule=match_rule, match_radius=match_radius, connectivity=connectivity,
                    edge_rule=edge_rule, walls=walls)
        if sequence:
            lx, ly = self.sizes[0]
            self.sizes = [(lx, ly)] * int(sequence)
            cfg = vd_config_init(lx, ly, threshold, polarity, stream, max_components, **opts)
            h = C.c_void_p()
            _check(lib().vd_batch_create_sequence(C.byref(cfg), int(sequence), C.byref(h)), "vd_batch_create_sequence")
            self.h = h
        else:
            per = options or [{}] * len(self.sizes)
            cfgs = [vd_config_init(lx, ly, threshold, polarity, stream, max_components, **{**opts, **o})
                    for (lx, ly), o in zip(self.sizes, per)]
            self.h = vd_batch_create(cfgs)

    def push(self, fields) -> None:
        _check(vd_batch_push(self.h, [f.data_ptr() for f in fields]), "vd_batch_push")

    def set_obstacles(self, i: int, mask) -> None:
        """mask: host array [Ly, Lx] of instance i, nonzero = obstacle site."""
        import numpy as np
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        _check(lib().vd_batch_set_obstacles(self.h, int(i), m.ctypes.data, m.shape[1]), "vd_batch_set_obstacles")

    def push_host_ptrs(self, host_ptrs) -> None:
        arr = (C.c_void_p * len(host_ptrs))(*[C.c_void_p(p) for p in host_ptrs])
        _check(lib().vd_batch_push_host(self.h, arr), "vd_batch_push_host")

    def stage_host_ptrs(self, host_ptrs) -> None:
        """Copy the next frames (host pointers) into the batch's spare input
        buffers on its copy stream (vd_batch_stage_host)."""
        arr = (C.c_void_p * len(host_ptrs))(*[C.c_void_p(p) for p in host_ptrs])
        _check(lib().vd_batch_stage_host(self.h, arr), "vd_batch_stage_host")

    def push_staged(self) -> None:
        _check(lib().vd_batch_push_staged(self.h), "vd_batch_push_staged")

    def changes_all(self) -> dict:
        """Every instance's results of the last push (vd_batch_get_changes_all):
        per-instance status and counts, and the packed change lists."""
        n = len(self.sizes)
        per = {k: np.zeros(n, np.int32) for k in ("status", "n_prev", "n_now", "n_breaking", "n_arising")}
        c = vd_batch_changes()
        for k, a in per.items():
            setattr(c, k, a.ctypes.data_as(C.POINTER(C.c_int32)))
        _check(lib().vd_batch_get_changes_all(self.h, C.byref(c)), "vd_batch_get_changes_all")
        brk = np.empty(c.total_breaking, np.uint64)
        brkp = np.empty(c.total_breaking, np.uint64)
        ari = np.empty(c.total_arising, np.uint64)
        act = np.empty(c.total_active, np.uint8)
        c.breaking = brk.ctypes.data_as(C.POINTER(C.c_uint64))
        c.breaking_prev = brkp.ctypes.data_as(C.POINTER(C.c_uint64))
        c.cap_breaking = len(brk)
        c.arising = ari.ctypes.data_as(C.POINTER(C.c_uint64))
        c.cap_arising = len(ari)
        c.active = act.ctypes.data_as(C.POINTER(C.c_uint8))
        c.cap_active = len(act)
        _check(lib().vd_batch_get_changes_all(self.h, C.byref(c)), "vd_batch_get_changes_all")
        return dict(per, breaking=brk, breaking_prev=brkp, arising=ari, active=act)

    def set_timing(self, on: bool) -> None:
        _check(lib().vd_batch_set_timing(self.h, int(bool(on))), "vd_batch_set_timing")

    def timing(self):
        """(per-stage ms since the last call, stage names, kernel launches, pushes)."""
        ms = (C.c_double * 16)()
        n, kl, nf = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().vd_batch_get_timing(self.h, ms, 16, C.byref(n), C.byref(kl), C.byref(nf)), "vd_batch_get_timing")
        names = [lib().vd_stage_name(i).decode() for i in range(n.value)]
        return list(ms[: n.value]), names, kl.value, nf.value

    def check_info(self) -> dict:
        """Checked build: see Detector.check_info."""
        c, k, x = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().vd_batch_debug_check_info(self.h, C.byref(c), C.byref(k), C.byref(x)),
               "vd_batch_debug_check_info")
        return dict(checked=bool(c.value), first_check=k.value, index=x.value)

    def force_check(self, check_id: int) -> None:
        _check(lib().vd_batch_debug_force_check(self.h, int(check_id)), "vd_batch_debug_force_check")

    def set_tuning(self, voronoi_patch: int = 0, bucket_pct: int = 100, ring0: int = 9,
                   graph_blocks: int | None = None) -> None:
        """Launch shapes of the batch (vd_batch_set_tuning); results are identical for every setting.
        graph_blocks None keeps the current graph-stage form."""
        gb = self.tuning()["graph_blocks"] if graph_blocks is None else int(graph_blocks)
        t = vd_tuning(int(voronoi_patch), int(bucket_pct), int(ring0), gb)
        _check(lib().vd_batch_set_tuning(self.h, C.byref(t)), "vd_batch_set_tuning")

    def tuning(self) -> dict:
        t = vd_tuning()
        _check(lib().vd_batch_get_tuning(self.h, C.byref(t)), "vd_batch_get_tuning")
        return dict(voronoi_patch=t.voronoi_patch, bucket_pct=t.bucket_pct, ring0=t.ring0,
                    graph_blocks=t.graph_blocks)

    def export_state(self, i: int) -> np.ndarray:
        """Checkpoint of instance i's last frame (vd_batch_export_state)."""
        n = C.c_int64()
        s = lib().vd_batch_export_state(self.h, int(i), None, 0, C.byref(n))
        if s != VD_ERR_CAPACITY:
            _check(s, "vd_batch_export_state")
        buf = np.empty(n.value, np.uint8)
        _check(lib().vd_batch_export_state(self.h, int(i), buf.ctypes.data_as(C.c_void_p), buf.size, C.byref(n)),
               "vd_batch_export_state")
        return buf

    def import_state(self, i: int, blob) -> None:
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().vd_batch_import_state(self.h, int(i), b.ctypes.data_as(C.c_void_p), b.size),
               "vd_batch_import_state")

    def push_subset(self, active, fields) -> None:
        _check(vd_batch_push_subset(self.h, list(active), [f.data_ptr() for f in fields]), "vd_batch_push_subset")

    def counts(self, i):
        s, K, E, f = vd_batch_get_counts(self.h, i)
        _check(s, "vd_batch_get_counts")
        return K, E, f

    def labels(self, i):
        lx, ly = self.sizes[i]
        return self._read("vd_batch_get_labels", i, np.int32, lx * ly).reshape(ly, lx)

    def owners(self, i):
        lx, ly = self.sizes[i]
        return self._read("vd_batch_get_owners", i, np.int32, lx * ly).reshape(ly, lx)

    def centroids(self, i):
        K, _, _ = self.counts(i)
        return self._read("vd_batch_get_centroids_q10", i, np.int32, K, 2).reshape(-1, 2)

    def edges(self, i):
        _, E, _ = self.counts(i)
        return self._read("vd_batch_get_edges", i, np.uint64, E)

    def changes(self, i) -> dict:
        K, E, _ = self.counts(i)
        cap = max(E, 1) * 2 + 16
        s, ch, brk, brkp, ari, act = _changes(lambda c: vd_batch_get_changes(self.h, i, c), K, cap)
        _check(s, "vd_batch_get_changes")
        return dict(frame=ch.frame_index, K_prev=ch.n_prev, K=ch.n_now, n_matched=ch.n_matched,
                    n_edges=ch.n_edges, breaking=brk[: ch.n_breaking].copy(),
                    breaking_prev=brkp[: ch.n_breaking].copy(), arising=ari[: ch.n_arising].copy(),
                    active=act[: ch.n_now].copy(), global_trigger=ch.global_trigger)

    def close(self):
        if getattr(self, "h", None):
            vd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def clock_ns() -> int:
    """The served form's host clock (vd_server_clock_ns), in ns."""
    t = C.c_int64()
    _check(lib().vd_server_clock_ns(C.byref(t)), "vd_server_clock_ns")
    return t.value


class Server:
    """Served form (vd_server_*): frames of many simulations, continuous batching.

    ``poll`` returns tuples (ticket, sim, status, t_arrival_ns, t_submit_ns,
    t_done_ns, n_bubbles, n_edges, n_breaking, n_arising)."""

    def __init__(self, sizes, budget_bytes: int, max_batch: int = 64, threshold: float = 0.5,
                 polarity: int = VD_ABOVE, stream: int | None = None, max_components: int = 0, options=None,
                 keep_changes: bool = False):
        """``options``: optional list of per-simulation dicts of config options
        (events, match_rule, match_radius, connectivity, edge_rule, walls)."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.threshold, self.polarity, self.max_components = threshold, polarity, max_components
        self.sizes = {}
        sizes = [(int(lx), int(ly)) for lx, ly in sizes]
        per = options or [{}] * len(sizes)
        cfgs = (vd_config * max(len(sizes), 1))(*[vd_config_init(lx, ly, threshold, polarity, stream, max_components,
                                                                 **o) for (lx, ly), o in zip(sizes, per)])
        h = C.c_void_p()
        _check(lib().vd_server_create(cfgs, len(sizes), int(budget_bytes), int(max_batch), C.c_void_p(stream),
                                      C.byref(h)), "vd_server_create")
        self.h = h
        for k, sz in enumerate(sizes):
            self.sizes[k] = sz
        self._done = (vd_server_done * 1024)()
        if keep_changes:
            self.keep_changes(True)

    def open_sim(self, size, **options) -> int:
        """Open one more simulation (vd_server_open_sim); returns its id."""
        lx, ly = int(size[0]), int(size[1])
        cfg = vd_config_init(lx, ly, self.threshold, self.polarity, self.stream, self.max_components, **options)
        sid = C.c_int32()
        _check(lib().vd_server_open_sim(self.h, C.byref(cfg), C.byref(sid)), "vd_server_open_sim")
        self.sizes[sid.value] = (lx, ly)
        return sid.value

    def close_sim(self, sim: int) -> None:
        _check(lib().vd_server_close_sim(self.h, int(sim)), "vd_server_close_sim")

    def keep_changes(self, on: bool = True) -> None:
        _check(lib().vd_server_keep_changes(self.h, int(bool(on))), "vd_server_keep_changes")

    def submit(self, sim: int, field, t_arrival_ns: int = 0) -> int:
        t = C.c_int64()
        _check(lib().vd_server_submit(self.h, int(sim), C.c_void_p(field.data_ptr()), int(t_arrival_ns), C.byref(t)),
               "vd_server_submit")
        return t.value

    def poll(self, wait: bool = False):
        n = C.c_int32()
        _check(lib().vd_server_poll(self.h, int(bool(wait)), self._done, 1024, C.byref(n)), "vd_server_poll")
        return [(d.ticket, d.sim, d.status, d.t_arrival_ns, d.t_submit_ns, d.t_done_ns, d.n_bubbles, d.n_edges,
                 d.n_breaking, d.n_arising) for d in self._done[: n.value]]

    def frame_changes(self, ticket: int, K: int) -> dict:
        """Changes of a frame retired by the last poll (vd_server_get_frame_changes)."""
        cap = 1 << 16
        s, ch, brk, brkp, ari, act = _changes(
            lambda c: lib().vd_server_get_frame_changes(self.h, int(ticket), C.byref(c)), K, cap)
        _check(s, "vd_server_get_frame_changes")
        return dict(frame=ch.frame_index, K_prev=ch.n_prev, K=ch.n_now, n_matched=ch.n_matched,
                    n_edges=ch.n_edges, breaking=brk[: ch.n_breaking].copy(),
                    breaking_prev=brkp[: ch.n_breaking].copy(), arising=ari[: ch.n_arising].copy(),
                    active=act[: ch.n_now].copy(), global_trigger=ch.global_trigger)

    def stats(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().vd_server_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "vd_server_stats")
        return dict(steps=a.value, frames_done=b.value, resident_bytes=c.value, queued=d.value)

    def labels(self, sim: int) -> np.ndarray:
        lx, ly = self.sizes[sim]
        out = np.empty(lx * ly, np.int32)
        n = C.c_int64()
        _check(lib().vd_server_get_labels(self.h, int(sim), out.ctypes.data_as(C.c_void_p), out.size, C.byref(n)),
               "vd_server_get_labels")
        return out.reshape(ly, lx)

    def changes(self, sim: int) -> dict:
        cap = 1 << 16
        s, ch, brk, brkp, ari, act = _changes(lambda c: lib().vd_server_get_changes(self.h, int(sim), C.byref(c)),
                                              1 << 22, cap)
        _check(s, "vd_server_get_changes")
        return dict(frame=ch.frame_index, K=ch.n_now, breaking=brk[: ch.n_breaking].copy(),
                    breaking_prev=brkp[: ch.n_breaking].copy(), arising=ari[: ch.n_arising].copy(),
                    active=act[: ch.n_now].copy())

    def export_state(self, sim: int) -> np.ndarray:
        n = C.c_int64()
        s = lib().vd_server_export_state(self.h, int(sim), None, 0, C.byref(n))
        if s != VD_ERR_CAPACITY:
            _check(s, "vd_server_export_state")
        buf = np.empty(n.value, np.uint8)
        _check(lib().vd_server_export_state(self.h, int(sim), buf.ctypes.data_as(C.c_void_p), buf.size,
                                            C.byref(n)), "vd_server_export_state")
        return buf

    def import_state(self, sim: int, blob) -> None:
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().vd_server_import_state(self.h, int(sim), b.ctypes.data_as(C.c_void_p), b.size),
               "vd_server_import_state")

    def close(self):
        if getattr(self, "h", None):
            lib().vd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
