"""CPU oracle of the detect pipeline (test infrastructure, not product code).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline
and reference arm) may import this package. It shares no code with the CUDA
path in ``paper_1607_00908_gb300/``; the two meet only on the seeded input
fields of ``paper_1607_00908_gb300.inputs``.
"""
from .detect import (  # noqa: F401
    OBSTACLE,
    OUTSIDE,
    Q,
    FRAME,
    Detector,
    EV_ACTIVE,
    EV_BOUNDARY,
    EV_BPOINT_NOW,
    EV_BPOINT_PAST,
    EV_BULK,
    adjacency,
    boundary_point,
    centroids_q10,
    classify_events,
    component_sums,
    delaunay_edges,
    flips,
    foreground,
    frame_gaps,
    incircle,
    label_components,
    make_keys,
    match_centroid,
    match_overlap,
    orient2d,
    owners,
    owners_at_points,
    owners_bruteforce,
    plaquette_diagonal,
    rdiv,
    split_keys,
    wide_components,
    vertex_edges,
    wrap,
    wrap_ax,
)
