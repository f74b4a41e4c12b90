"""Brute-force periodic Delaunay triangulation for pinning the oracle's edge step.

Independent of ``oracle/``: exact empty-circle test with Python integers on the
3x3 periodic tiling of a point set on a torus, O(n^4) in the worst case but
restricted to local triples. Used only on tiny generic configurations.
"""
from __future__ import annotations

import itertools


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _incircle(a, b, c, d):
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            + (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def _circumcentre(a, b, c):
    ax, ay = a
    bx, by = b
    cx, cy = c
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay)
          + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx)
          + (cx * cx + cy * cy) * (bx - ax)) / d
    return ux, uy


def periodic_delaunay(points, W, H, radius):
    """Delaunay triangles of integer points on a W x H torus.

    points: list of (x, y) ints in [0, W) x [0, H). ``radius`` bounds the
    distance from a central vertex to the other two vertices of the triangles
    considered (must exceed every Delaunay edge length).

    Returns (edges, triangles, min_incircle_margin, min_dual_length, dual_of):
      edges      set of (i, j), i < j, label pairs of Delaunay edges
      triangles  list of ((i, oi), (j, oj), (k, ok)) with vertex 0 central
      margin     smallest |incircle| seen over the emptiness checks of the
                 accepted triangles against all other tiled points (0 means a
                 cocircular, non-generic configuration)
      dual       smallest length of a Voronoi edge dual to a Delaunay edge
      dual_of    dict label pair -> shortest dual Voronoi edge length among the
                 periodic edges that carry that pair
    """
    n = len(points)
    tiled = []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for i, (x, y) in enumerate(points):
                tiled.append((i, (ox, oy), (x + ox * W, y + oy * H)))
    r2 = radius * radius
    tris = []
    margin = None
    for i, (x, y) in enumerate(points):
        a = (x, y)
        near = [t for t in tiled
                if (t[2][0] - x) ** 2 + (t[2][1] - y) ** 2 <= r2 and not (t[0] == i and t[1] == (0, 0))]
        for (j, oj, b), (k, ok, c) in itertools.combinations(near, 2):
            o = _orient(a, b, c)
            if o == 0:
                continue
            if o < 0:
                (j, oj, b), (k, ok, c) = (k, ok, c), (j, oj, b)
            empty = True
            local_min = None
            for (m, om, d) in tiled:
                if (m == i and om == (0, 0)) or (m == j and om == oj) or (m == k and om == ok):
                    continue
                v = _incircle(a, b, c, d)
                if v > 0:
                    empty = False
                    break
                av = -v
                local_min = av if local_min is None else min(local_min, av)
            if empty:
                tris.append(((i, (0, 0), a), (j, oj, b), (k, ok, c)))
                if local_min is not None:
                    margin = local_min if margin is None else min(margin, local_min)
    edges = set()
    for t in tris:
        for (p, _, _), (q, _, _) in itertools.combinations(t, 2):
            if p != q:
                edges.add((min(p, q), max(p, q)))
    # dual Voronoi edge lengths: for each edge (central u, tiled v), the two
    # triangles incident to u that contain v
    dual = None
    dual_of = {}
    for t in tris:
        u = t[0]
        for v in (t[1], t[2]):
            adj = [s for s in tris if s[0][0] == u[0] and any(
                (w[0] == v[0] and w[1] == v[1]) for w in s[1:])]
            if len(adj) == 2:
                c1 = _circumcentre(*[w[2] for w in adj[0]])
                c2 = _circumcentre(*[w[2] for w in adj[1]])
                dl = ((c1[0] - c2[0]) ** 2 + (c1[1] - c2[1]) ** 2) ** 0.5
                dual = dl if dual is None else min(dual, dl)
                key = (min(u[0], v[0]), max(u[0], v[0]))
                dual_of[key] = min(dual_of.get(key, dl), dl)
    return edges, tris, (margin or 0), (dual if dual is not None else 0.0), dual_of
