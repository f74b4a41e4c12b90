"""CPU oracle for the detect pipeline: plain, slow, and written to be checked by eye.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm
of ``bench.py`` may call it. It shares no code with the CUDA path.

Every function states the passage of the paper it follows (M. Bernaschi,
M. Lulli, M. Sbragaglia, "GPU Based Detection of Topological Changes in Voronoi
Diagrams", arXiv:1607.00908). Where the paper is silent or ambiguous the
reading taken is stated in the docstring. All arithmetic on the path is
integer (int64, or Python integers for the incircle determinant), so results
are exact and the GPU must match them bit for bit.

Library primitives used as single steps: ``scipy.ndimage.label`` (connected
components on the open rectangle), ``numpy.unique`` / sorting, and
``scipy.spatial.cKDTree`` (exact k-nearest-neighbour search; its float64
arithmetic is exact for the integer fixed-point coordinates used here, and
ties are resolved in integers afterwards). ``owners_bruteforce`` is the
literal definition and pins ``owners``.

``vertex_edges`` (the paper's frame / inner-frame link rule, an option)
follows a reading of figures that are lost. It is pinned to geometry -- the
periodic Delaunay triangulation on generic point sets, a triangulation on dense
random sets, hand-counted pathological colourings and ties -- but not to the
authors' code, and the pins do not decide the orientation of its quarter turns
(the mirror-image reading passes them too).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage
from scipy.spatial import cKDTree

#: Fixed-point scale of centroids: 1/1024 site.
Q = 1024


# ----------------------------------------------------------------------------
# Small integer helpers
# ----------------------------------------------------------------------------

def wrap(d, L):
    """Minimum-image displacement on a ring of length L: ((d + L//2) mod L) - L//2.

    Result lies in [-(L//2), L - L//2). Works elementwise on int64 arrays and on
    Python ints (both use floor modulo).
    """
    h = L // 2
    return ((d + h) % L) - h


def wrap_ax(d, L, periodic: bool):
    """Displacement along one axis: minimum image when the axis is periodic,
    plain difference when it is bounded by walls."""
    return wrap(d, L) if periodic else d


#: owner of an obstacle site (the paper's MAXLINK colour) and, in frame
#: tests, of a neighbour that lies beyond a wall
OBSTACLE, OUTSIDE = -2, -3


def rdiv(p, q):
    """Round-half-up integer division p/q for q > 0: floor((2p + q) / (2q))."""
    return (2 * p + q) // (2 * q)


# ----------------------------------------------------------------------------
# Section 3.1: threshold and cluster labelling
# ----------------------------------------------------------------------------

def foreground(F, theta: float = 0.5, polarity: int = 1) -> np.ndarray:
    """Spin variable of Section 3.1 as a boolean: site belongs to a bubble.

    The paper calls a site part of a bubble when the field is *below* the
    threshold; the workloads here mark droplets by values *above* it. Reading:
    ``polarity=+1`` means F > theta (strict), ``polarity=-1`` means F < theta.
    Comparisons are done in float32, and NaN is never foreground.
    """
    F = np.asarray(F, dtype=np.float32)
    t = np.float32(theta)
    return (F > t) if polarity > 0 else (F < t)


def _neighbour_offsets(connectivity: int):
    if connectivity == 4:
        return [(1, 0), (0, 1)]
    if connectivity == 8:
        return [(1, 0), (0, 1), (1, 1), (1, -1)]
    raise ValueError("connectivity must be 4 or 8")


def label_components(fg: np.ndarray, connectivity: int = 4, periodic=(True, True)):
    """Periodic connected-component labels with canonical ids (Section 3.1).

    Bubbles are maximal sets of foreground sites connected through lattice
    neighbours; the domain is a torus (both axes periodic). Reading: 4-neighbour
    connectivity by default (the Ising cluster-labelling analogy of Section 3.1),
    8 as an option. The paper fixes no label values; here a component's id is
    the rank of its smallest linear index y*Lx + x among all components, so ids
    run 0..K-1 in raster order of first sites. Background is -1. An axis that
    is not periodic (walls, the paper's channel) joins nothing across its seam.

    Returns (labels int32 [Ly, Lx], K).
    """
    fg = np.asarray(fg, dtype=bool)
    Ly, Lx = fg.shape
    struct = ndimage.generate_binary_structure(2, 1 if connectivity == 4 else 2)
    raw, npieces = ndimage.label(fg, structure=struct)
    if npieces == 0:
        return np.full((Ly, Lx), -1, dtype=np.int32), 0
    # Pieces of the open rectangle that touch across a periodic seam are the
    # same component: collect every neighbour pair (with wrap) whose raw labels
    # differ and join them with a union-find.
    parent = list(range(npieces + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    pairs = set()
    xs = np.arange(Lx)[None, :]
    ys = np.arange(Ly)[:, None]
    for dx, dy in _neighbour_offsets(connectivity):
        nb = np.roll(np.roll(raw, -dy, axis=0), -dx, axis=1)   # raw at (x+dx, y+dy)
        m = (raw > 0) & (nb > 0) & (raw != nb)
        if not periodic[0]:
            m &= (xs + dx >= 0) & (xs + dx < Lx)
        if not periodic[1]:
            m &= (ys + dy >= 0) & (ys + dy < Ly)
        if m.any():
            a = raw[m].astype(np.int64)
            b = nb[m].astype(np.int64)
            pairs.update(zip(np.minimum(a, b).tolist(), np.maximum(a, b).tolist()))
    for a, b in pairs:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(npieces + 1)], dtype=np.int64)
    # smallest linear index of each piece, then of each merged component
    flat = raw.ravel()
    ids, first = np.unique(flat, return_index=True)
    first_of_piece = np.full(npieces + 1, np.iinfo(np.int64).max, dtype=np.int64)
    first_of_piece[ids] = first
    first_of_root = np.full(npieces + 1, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(first_of_root, roots[1:], first_of_piece[1:])
    comp_roots = np.unique(roots[1:])
    order = np.argsort(first_of_root[comp_roots], kind="stable")
    canon = np.full(npieces + 1, -1, dtype=np.int64)
    rank_of_root = np.empty(npieces + 1, dtype=np.int64)
    rank_of_root[comp_roots[order]] = np.arange(comp_roots.size)
    canon[1:] = rank_of_root[roots[1:]]
    labels = canon[raw].astype(np.int32)
    return labels, int(comp_roots.size)


# ----------------------------------------------------------------------------
# Section 3.1: size and centre of mass
# ----------------------------------------------------------------------------

def component_sums(labels: np.ndarray, K: int, periodic=(True, True)):
    """Per component: root site r, size n, and Sx, Sy = sums of wrap(x - x_r), wrap(y - y_r).

    Section 3.1 counts the sites of each bubble and sums their x and y
    coordinates separately. On the torus the coordinates are taken as
    minimum-image displacements from the component's first site r (smallest
    linear index), which is this implementation's reading of a periodic centre
    of mass. Returns int64 arrays (xr, yr, n, Sx, Sy), each of length K.
    """
    Ly, Lx = labels.shape
    flat = labels.ravel().astype(np.int64)
    idx = np.flatnonzero(flat >= 0)
    lab = flat[idx]
    first = np.full(K, Lx * Ly, dtype=np.int64)
    np.minimum.at(first, lab, idx)
    xr = first % Lx
    yr = first // Lx
    x = idx % Lx
    y = idx // Lx
    dx = wrap_ax(x - xr[lab], Lx, periodic[0])
    dy = wrap_ax(y - yr[lab], Ly, periodic[1])
    n = np.bincount(lab, minlength=K).astype(np.int64)
    Sx = np.zeros(K, dtype=np.int64)
    Sy = np.zeros(K, dtype=np.int64)
    np.add.at(Sx, lab, dx)
    np.add.at(Sy, lab, dy)
    return xr, yr, n, Sx, Sy


def centroids_q10(labels: np.ndarray, K: int, periodic=(True, True)) -> np.ndarray:
    """Centre of mass of each bubble in 1/1024-site fixed point (Section 3.1).

    c = x_r + Sx / n per axis, with the division rounded half up in units of
    1/1024 site and the result taken modulo the lattice:
    cx = (1024*x_r + rdiv(1024*Sx, n)) mod (1024*Lx), likewise cy.
    Returns int64 array [K, 2] of (cx, cy).
    """
    Ly, Lx = labels.shape
    if K == 0:
        return np.zeros((0, 2), dtype=np.int64)
    xr, yr, n, Sx, Sy = component_sums(labels, K, periodic)
    cx = np.mod(Q * xr + rdiv(Q * Sx, n), Q * Lx)
    cy = np.mod(Q * yr + rdiv(Q * Sy, n), Q * Ly)
    return np.stack([cx, cy], axis=1).astype(np.int64)


def wide_components(labels: np.ndarray, K: int, periodic=(True, True)) -> np.ndarray:
    """Components too wide for a compact centre on the torus (Section 3.1 with
    the minimum-image reading of ``component_sums``): along a periodic axis the
    minimum-image displacements of the sites from the first site span half the
    period or more (one that winds around the torus spans all of it). The
    centroid formula still applies to them, but its result is then a
    convention, not the centre of a blob. Displacements along a bounded axis
    are plain, so walls never make a component wide. Returns bool [K].
    """
    Ly, Lx = labels.shape
    out = np.zeros(K, dtype=bool)
    if K == 0:
        return out
    flat = labels.ravel().astype(np.int64)
    idx = np.flatnonzero(flat >= 0)
    lab = flat[idx]
    first = np.full(K, Lx * Ly, dtype=np.int64)
    np.minimum.at(first, lab, idx)
    axes = ((idx % Lx, first % Lx, Lx, periodic[0]), (idx // Lx, first // Lx, Ly, periodic[1]))
    for c, c_r, L, per in axes:
        if not per:
            continue
        d = wrap(c - c_r[lab], L)
        lo = np.full(K, L, dtype=np.int64)
        hi = np.full(K, -L, dtype=np.int64)
        np.minimum.at(lo, lab, d)
        np.maximum.at(hi, lab, d)
        out |= 2 * (hi - lo + 1) >= L
    return out


# ----------------------------------------------------------------------------
# Section 3.2.1: digital Voronoi tessellation
# ----------------------------------------------------------------------------

def _site_grid(Lx: int, Ly: int):
    y, x = np.divmod(np.arange(Lx * Ly, dtype=np.int64), Lx)
    return x, y


def sq_dist_q10(sx, sy, cx, cy, Lx: int, Ly: int, periodic=(True, True)):
    """Exact squared distance between Q10 points (int64), minimum image on
    periodic axes."""
    dx = wrap_ax(sx - cx, Q * Lx, periodic[0])
    dy = wrap_ax(sy - cy, Q * Ly, periodic[1])
    return dx * dx + dy * dy


def owners_bruteforce(cq: np.ndarray, Lx: int, Ly: int, sites=None, periodic=(True, True)) -> np.ndarray:
    """Digital Voronoi colouring, literally as in Section 3.2.1.

    Every site (foreground or not) takes the label of the nearest centre of
    mass by squared Euclidean distance (no square root). Distances are exact
    int64 in 1/1024-site units with minimum image on the torus; the site (x, y)
    sits at (1024x, 1024y). The paper leaves ties open; here a tie goes to the
    smallest label (np.argmin returns the first minimum). With no centres every
    owner is -1. ``sites`` optionally restricts the evaluation to an int64 array
    of linear indices.
    """
    K = cq.shape[0]
    if sites is None:
        x, y = _site_grid(Lx, Ly)
    else:
        sites = np.asarray(sites, dtype=np.int64)
        y, x = np.divmod(sites, Lx)
    out = np.full(x.shape[0], -1, dtype=np.int32)
    if K == 0:
        return out if sites is not None else out.reshape(Ly, Lx)
    sx = Q * x
    sy = Q * y
    cx = cq[:, 0].astype(np.int64)
    cy = cq[:, 1].astype(np.int64)
    chunk = max(1, 4_000_000 // K)
    for s in range(0, x.shape[0], chunk):
        d2 = sq_dist_q10(sx[s:s + chunk, None], sy[s:s + chunk, None],
                         cx[None, :], cy[None, :], Lx, Ly, periodic)
        out[s:s + chunk] = np.argmin(d2, axis=1)
    return out if sites is not None else out.reshape(Ly, Lx)


def owners_at_points(cq: np.ndarray, Lx: int, Ly: int, px, py, periodic=(True, True)) -> np.ndarray:
    """Voronoi colour of arbitrary points in 1/1024-site units (the colouring
    rule of Section 3.2.1 applied to points that need not be lattice sites,
    such as the inner-frame points of Section 3.2.2): the label of the nearest
    centre by exact int64 squared distance, minimum image on periodic axes,
    ties to the smallest label; -1 when there are no centres."""
    px = np.asarray(px, dtype=np.int64).ravel()
    py = np.asarray(py, dtype=np.int64).ravel()
    K = cq.shape[0]
    out = np.full(px.shape[0], -1, dtype=np.int32)
    if K == 0 or px.size == 0:
        return out
    cx = cq[:, 0].astype(np.int64)
    cy = cq[:, 1].astype(np.int64)
    chunk = max(1, 4_000_000 // K)
    for s in range(0, px.shape[0], chunk):
        d2 = sq_dist_q10(px[s:s + chunk, None], py[s:s + chunk, None], cx[None, :], cy[None, :], Lx, Ly, periodic)
        out[s:s + chunk] = np.argmin(d2, axis=1)
    return out


def owners(cq: np.ndarray, Lx: int, Ly: int, workers: int = 1) -> np.ndarray:
    """Same result as ``owners_bruteforce``, with a k-d tree as the search step.

    The tree (periodic box of 1024*Lx by 1024*Ly) returns the k = 4 nearest
    centres of every site. Its float64 distances are exact here: coordinates are
    integers below 2**23 and squared distances below 2**45. The exact int64
    squared distances of those k candidates are then recomputed, and the owner
    is the smallest label among the candidates at the minimum. Where the k-th
    candidate also sits at the minimum (a tie that may extend past k), the site
    is resolved by the brute-force definition.
    """
    K = cq.shape[0]
    if K == 0:
        return np.full((Ly, Lx), -1, dtype=np.int32)
    x, y = _site_grid(Lx, Ly)
    sx = Q * x
    sy = Q * y
    k = min(4, K)
    tree = cKDTree(cq.astype(np.float64), boxsize=[float(Q * Lx), float(Q * Ly)])
    pts = np.stack([sx, sy], axis=1).astype(np.float64)
    _, ind = tree.query(pts, k=k, workers=workers)
    ind = ind.reshape(-1, k).astype(np.int64)
    cx = cq[:, 0].astype(np.int64)
    cy = cq[:, 1].astype(np.int64)
    d2 = sq_dist_q10(sx[:, None], sy[:, None], cx[ind], cy[ind], Lx, Ly)
    best = d2.min(axis=1)
    at_best = d2 == best[:, None]
    cand = np.where(at_best, ind, np.iinfo(np.int64).max)
    out = cand.min(axis=1).astype(np.int32)
    if k < K:
        unsure = np.flatnonzero(at_best[:, k - 1])
        if unsure.size:
            out[unsure] = owners_bruteforce(cq, Lx, Ly, sites=unsure)
    return out.reshape(Ly, Lx)


# ----------------------------------------------------------------------------
# Section 3.2.2: Delaunay edges from the digital Voronoi colouring
# ----------------------------------------------------------------------------

def orient2d(a, b, c) -> int:
    """Twice the signed area of triangle abc (Python ints, exact)."""
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def incircle(a, b, c, d) -> int:
    """In-circle determinant (Python ints, exact): > 0 iff d lies inside the
    circle through a, b, c when a, b, c are counter-clockwise."""
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            + (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def _sign(v: int) -> int:
    return (v > 0) - (v < 0)


def plaquette_diagonal(A: int, B: int, C: int, D: int, cq: np.ndarray,
                       Lx: int, Ly: int, periodic=(True, True)):
    """Diagonal link of a 2x2 plaquette whose four owners are pairwise distinct.

    The plaquette's sites (x,y), (x+1,y), (x+1,y+1), (x,y+1) carry owners A, B,
    C, D in cyclic order, so four Voronoi cells meet inside it and one of the
    diagonals A-C or B-D is a Delaunay edge (Section 3.2.2, the second-nearest-
    neighbour case, whose fifth condition decides which diagonal to keep). The
    figure that fixes the paper's inner-frame point is lost, so the decision is
    taken here by the exact Delaunay criterion on the four centres, unwrapped by
    minimum image around A: s = sign(incircle(a,b,c,d)) * sign(orient(a,b,c)).
    s > 0 (d inside the circle of a, b, c) keeps B-D, s < 0 keeps A-C, and an
    exact tie (s = 0) keeps the diagonal whose smaller label is smaller.
    Returns the kept pair (lo, hi).
    """
    ax, ay = int(cq[A, 0]), int(cq[A, 1])

    def unwrapped(i):
        return (ax + int(wrap_ax(int(cq[i, 0]) - ax, Q * Lx, periodic[0])),
                ay + int(wrap_ax(int(cq[i, 1]) - ay, Q * Ly, periodic[1])))

    a = (ax, ay)
    b, c, d = unwrapped(B), unwrapped(C), unwrapped(D)
    s = _sign(incircle(a, b, c, d)) * _sign(orient2d(a, b, c))
    if s > 0 or (s == 0 and min(B, D) < min(A, C)):
        return (min(B, D), max(B, D))
    return (min(A, C), max(A, C))


def delaunay_edges(owner: np.ndarray, cq: np.ndarray, periodic=(True, True)) -> np.ndarray:
    """Delaunay edge set of the digital Voronoi diagram, as sorted uint64 keys.

    Section 3.2.2 reads the adjacency of Voronoi cells off the colours of
    neighbouring sites. Reading taken here (the paper's vertex/inner-frame rule
    depends on a lost figure): two labels are linked when

    (i)  a site and its +x or +y neighbour (periodic) have different owners, or
    (ii) a 2x2 plaquette carries four pairwise distinct owners; then the
         diagonal chosen by ``plaquette_diagonal`` is linked.

    A link {a, b} is stored once as the key (min << 32) | max; the result is
    sorted and unique (the "compressed adjacency" of Section 3.2.2). Pairs and
    plaquettes that would cross a wall (a bounded axis), and sites of
    obstacles (negative owners), give no link.
    """
    Ly, Lx = owner.shape
    A = owner.astype(np.int64)
    B = np.roll(A, -1, axis=1)                    # owner at (x+1, y)
    D = np.roll(A, -1, axis=0)                    # owner at (x, y+1)
    C = np.roll(B, -1, axis=0)                    # owner at (x+1, y+1)
    inx = np.ones((Ly, Lx), dtype=bool)
    iny = np.ones((Ly, Lx), dtype=bool)
    if not periodic[0]:
        inx[:, Lx - 1] = False                    # (x+1) lies beyond the wall
    if not periodic[1]:
        iny[Ly - 1, :] = False
    keys = []
    for P, R, inside in ((A, B, inx), (A, D, iny)):
        m = (P != R) & inside & (P >= 0) & (R >= 0)
        lo = np.minimum(P[m], R[m])
        hi = np.maximum(P[m], R[m])
        keys.append((lo << 32) | hi)
    four = (A != B) & (A != C) & (A != D) & (B != C) & (B != D) & (C != D)
    four &= inx & iny & (A >= 0) & (B >= 0) & (C >= 0) & (D >= 0)
    diag = []
    for ia, ib, ic, id_ in zip(A[four].tolist(), B[four].tolist(),
                               C[four].tolist(), D[four].tolist()):
        lo, hi = plaquette_diagonal(ia, ib, ic, id_, cq, Lx, Ly, periodic)
        diag.append((lo << 32) | hi)
    keys.append(np.array(diag, dtype=np.int64))
    allk = np.concatenate(keys) if keys else np.zeros(0, dtype=np.int64)
    return np.unique(allk).astype(np.uint64)


# ----------------------------------------------------------------------------
# Section 3.2.2, the paper's own link rule: vertex sites of the digital
# Voronoi diagram and the frame / inner-frame conditions (option)
# ----------------------------------------------------------------------------

#: the frame of a site: its eight neighbours in counter-clockwise order,
#: starting at +x (spx, spxpy, spy, spymx, smx, smxmy, smy, smypx)
FRAME = ((1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1))


def _shifted(owner: np.ndarray, dx: int, dy: int, periodic=(True, True)) -> np.ndarray:
    """owner at (x+dx, y+dy); OUTSIDE where that crosses a wall."""
    Ly, Lx = owner.shape
    out = np.roll(np.roll(owner.astype(np.int64), -dy, axis=0), -dx, axis=1)
    if not periodic[0]:
        xs = np.arange(Lx)[None, :] + dx
        out = np.where((xs < 0) | (xs >= Lx), OUTSIDE, out)
    if not periodic[1]:
        ys = np.arange(Ly)[:, None] + dy
        out = np.where((ys < 0) | (ys >= Ly), OUTSIDE, out)
    return out


def frame_gaps(owner: np.ndarray, periodic=(True, True)) -> np.ndarray:
    """Number of colour changes between consecutive sites of each frame. At a
    wall the frame keeps only the neighbours inside the domain (taken in the
    same cyclic order); an obstacle neighbour counts with its MAXLINK colour."""
    fr = [_shifted(owner, dx, dy, periodic) for dx, dy in FRAME]
    Ly, Lx = owner.shape
    gaps = np.zeros((Ly, Lx), dtype=np.int64)
    # previous in-domain member of each frame, starting from the last one
    prev = np.full((Ly, Lx), OUTSIDE, dtype=np.int64)
    for i in range(8):
        prev = np.where(fr[i] != OUTSIDE, fr[i], prev)
    for i in range(8):
        inside = fr[i] != OUTSIDE
        gaps += (inside & (fr[i] != prev)).astype(np.int64)
        prev = np.where(inside, fr[i], prev)
    return gaps


def vertex_edges(owner: np.ndarray, cq: np.ndarray, periodic=(True, True)) -> np.ndarray:
    """Links read at the vertex sites of the digital Voronoi diagram (Section
    3.2.2, the paper's frame rule), as sorted uint64 keys. The figures that
    define the inner frame and the pathological colourings are lost, so the
    readings below are checked against geometry (Delaunay triangulations,
    hand-counted colourings), not against the authors' code; the mirror-image
    reading (quarter turns clockwise) passes the same checks.

    Readings: a vertex site has three or more colour changes around its frame
    (two: a cell edge, none: a cell interior). On a periodic lattice without
    obstacles no colour is MAXLINK. With e1 one of +x, +y, -x, -y and e2 = e1
    turned a quarter counter-clockwise, the conditions written for spx and
    spxpy are applied to the four quarter turns:

    * first neighbour k+e1 is linked to k when its colour differs from k's and
      C(k+e2) != C(k+e1-e2) (the long-diagonal pathology);
    * second neighbour k+e1+e2 is linked to k when its colour differs from
      k's, C(k+e2) != C(k+e1-e2), C(k+e2) != C(k+e1) (the short diagonal),
      and the inner-frame point -- read as the centre of the plaquette,
      k + (e1+e2)/2 -- takes k's colour or the neighbour's. Its colour C(a_k)
      is its Voronoi colour, as for every point of the stencil: the nearest
      centre over all centres, by the exact rule of Section 3.2.1
      (``owners_at_points``). A centre whose cell holds the plaquette centre
      but no lattice site therefore blocks the diagonal.

    Walls truncate the frame (neighbours beyond them leave it) and obstacle
    sites carry the MAXLINK colour: neither is ever linked, nor is a site that
    is itself an obstacle.
    """
    Ly, Lx = owner.shape
    own = owner.astype(np.int64)

    def at(dx, dy):
        return _shifted(own, dx, dy, periodic)

    vert = (frame_gaps(own, periodic) >= 3) & (own >= 0)
    keys = []
    turns = ((1, 0), (0, 1), (-1, 0), (0, -1))
    for e1x, e1y in turns:
        e2x, e2y = -e1y, e1x
        X = at(e1x, e1y)
        ok = vert & (X >= 0) & (X != own) & (at(e2x, e2y) != at(e1x - e2x, e1y - e2y))
        keys.append(make_keys(own[ok], X[ok]).astype(np.int64))
    for e1x, e1y in turns:
        e2x, e2y = -e1y, e1x
        X = at(e1x + e2x, e1y + e2y)
        A1, A2, A3 = at(e1x, e1y), at(e2x, e2y), at(e1x - e2x, e1y - e2y)
        ok = vert & (X >= 0) & (X != own) & (A2 != A3) & (A2 != A1)
        ys, xs = np.nonzero(ok)
        if xs.size == 0:
            continue
        px = (Q * xs + (Q // 2) * (e1x + e2x)) % (Q * Lx)
        py = (Q * ys + (Q // 2) * (e1y + e2y)) % (Q * Ly)
        kk, xx = own[ys, xs], X[ys, xs]
        # colour of the inner-frame point: its exact Voronoi owner
        ca = owners_at_points(cq, Lx, Ly, px, py, periodic)
        sel = (ca == kk) | (ca == xx)
        keys.append(make_keys(kk[sel], xx[sel]).astype(np.int64))
    allk = np.concatenate(keys) if keys else np.zeros(0, dtype=np.int64)
    return np.unique(allk).astype(np.uint64)


# ----------------------------------------------------------------------------
# Section 3.2.3: isomorphism between past and now labels
# ----------------------------------------------------------------------------

def match_overlap(lab_prev: np.ndarray, lab_now: np.ndarray, K_prev: int, K_now: int):
    """Label isomorphism Phi_{P->N} by mutual best overlap (Section 3.2.3).

    The paper obtains Phi by comparing the two sets of centres of mass of
    frames a short time apart, and excludes labels where the map is not
    injective (a bubble vanished) or a now-label has no partner (a bubble
    appeared). Reading used here: H(p, n) counts sites labelled p in the past
    frame and n now. best_n(p) = argmax_n H(p, n) (ties to the smallest n),
    best_p(n) likewise, and Phi(p) = n exactly when the choice is mutual;
    every other label is unmatched (-1). Returns (phi [K_prev], inv [K_now]).
    """
    phi = np.full(K_prev, -1, dtype=np.int32)
    inv = np.full(K_now, -1, dtype=np.int32)
    m = (lab_prev >= 0) & (lab_now >= 0)
    if K_prev == 0 or K_now == 0 or not m.any():
        return phi, inv
    keys = lab_prev[m].astype(np.int64) * K_now + lab_now[m].astype(np.int64)
    uk, cnt = np.unique(keys, return_counts=True)
    p = uk // K_now
    n = uk % K_now
    # best n for each p: largest count, then smallest n
    o = np.lexsort((n, -cnt, p))
    first = np.ones(o.size, dtype=bool)
    first[1:] = p[o][1:] != p[o][:-1]
    best_n = np.full(K_prev, -1, dtype=np.int64)
    best_n[p[o][first]] = n[o][first]
    # best p for each n: largest count, then smallest p
    o = np.lexsort((p, -cnt, n))
    first = np.ones(o.size, dtype=bool)
    first[1:] = n[o][1:] != n[o][:-1]
    best_p = np.full(K_now, -1, dtype=np.int64)
    best_p[n[o][first]] = p[o][first]
    pp = np.flatnonzero(best_n >= 0)
    mutual = best_p[best_n[pp]] == pp
    phi[pp[mutual]] = best_n[pp[mutual]]
    inv[best_n[pp[mutual]]] = pp[mutual]
    return phi, inv


def _nearest(q: np.ndarray, c: np.ndarray, Lx: int, Ly: int, R2: int, periodic=(True, True)) -> np.ndarray:
    """For every row of q (Q10 centres) the index of the nearest row of c by
    minimum-image squared distance (int64), ties to the smallest index, or -1
    when the nearest is farther than sqrt(R2). Brute force in chunks."""
    out = np.full(q.shape[0], -1, dtype=np.int64)
    if q.shape[0] == 0 or c.shape[0] == 0:
        return out
    cx = c[:, 0].astype(np.int64)
    cy = c[:, 1].astype(np.int64)
    for i0 in range(0, q.shape[0], 512):
        qx = q[i0:i0 + 512, 0].astype(np.int64)[:, None]
        qy = q[i0:i0 + 512, 1].astype(np.int64)[:, None]
        dx = wrap_ax(cx[None, :] - qx, Q * Lx, periodic[0])
        dy = wrap_ax(cy[None, :] - qy, Q * Ly, periodic[1])
        d = dx * dx + dy * dy
        j = np.argmin(d, axis=1)          # first index of the minimum: ties to the smallest
        dmin = d[np.arange(d.shape[0]), j]
        out[i0:i0 + 512] = np.where(dmin <= R2, j, -1)
    return out


def match_centroid(cq_prev: np.ndarray, cq_now: np.ndarray, Lx: int, Ly: int, radius: int,
                   periodic=(True, True)):
    """Label isomorphism Phi_{P->N} from the two sets of centres (Section 3.2.3,
    the paper's kinematic comparison of frames a short time apart).

    Reading: best_n(p) = the now centre nearest to past centre p, best_p(n)
    the past centre nearest to now centre n (minimum-image squared distance in
    1/1024 sites, ties to the smallest label), each only within `radius`
    sites. Phi(p) = n exactly when the choice is mutual, which keeps the map
    injective; every other label is unmatched (-1), as the paper excludes
    vanishing and appearing bubbles. Returns (phi [K_prev], inv [K_now]).
    """
    cq_prev = np.asarray(cq_prev, dtype=np.int64).reshape(-1, 2)
    cq_now = np.asarray(cq_now, dtype=np.int64).reshape(-1, 2)
    K_prev, K_now = cq_prev.shape[0], cq_now.shape[0]
    phi = np.full(K_prev, -1, dtype=np.int32)
    inv = np.full(K_now, -1, dtype=np.int32)
    R2 = (Q * int(radius)) ** 2
    best_n = _nearest(cq_prev, cq_now, Lx, Ly, R2, periodic)
    best_p = _nearest(cq_now, cq_prev, Lx, Ly, R2, periodic)
    for p in range(K_prev):
        n = int(best_n[p])
        if n >= 0 and int(best_p[n]) == p:
            phi[p] = n
            inv[n] = p
    return phi, inv


# ----------------------------------------------------------------------------
# Sections 3.2.3-3.2.4: translation, comparison, breaking and arising links
# ----------------------------------------------------------------------------

def split_keys(E: np.ndarray):
    E = np.asarray(E, dtype=np.uint64)
    return (E >> np.uint64(32)).astype(np.int64), (E & np.uint64(0xFFFFFFFF)).astype(np.int64)


def make_keys(a, b) -> np.ndarray:
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    return ((lo << 32) | hi).astype(np.uint64)


def flips(E_prev: np.ndarray, E_now: np.ndarray, phi: np.ndarray, inv: np.ndarray):
    """Breaking and arising links between two triangulations (Sections 3.2.3-3.2.4).

    Translation: every past link {a, b} with both ends matched becomes
    {Phi(a), Phi(b)} in now-labels. Links with an unmatched end, and now-links
    touching a label outside Phi's image, are excluded (appearing or vanishing
    bubbles). A link present only in the translated past set is *breaking*,
    one present only in the now set is *arising*. Both lists are sorted by
    now-key; each breaking link also carries its past-label key. ``active`` is
    the local trigger: 1 for every now-label at an end of a flip.

    Returns dict(breaking, breaking_prev, arising, active, global_trigger).
    """
    K_now = inv.shape[0]
    a, b = split_keys(E_prev)
    keep = (phi[a] >= 0) & (phi[b] >= 0) if a.size else np.zeros(0, dtype=bool)
    EPt = np.unique(make_keys(phi[a[keep]], phi[b[keep]])) if keep.any() else np.zeros(0, np.uint64)
    na, nb = split_keys(E_now)
    keepn = (inv[na] >= 0) & (inv[nb] >= 0) if na.size else np.zeros(0, dtype=bool)
    ENt = np.asarray(E_now, dtype=np.uint64)[keepn]
    breaking = np.setdiff1d(EPt, ENt).astype(np.uint64)
    arising = np.setdiff1d(ENt, EPt).astype(np.uint64)
    ba, bb = split_keys(breaking)
    breaking_prev = make_keys(inv[ba], inv[bb]) if breaking.size else np.zeros(0, np.uint64)
    active = np.zeros(K_now, dtype=np.uint8)
    for E in (breaking, arising):
        x, y = split_keys(E)
        active[x] = 1
        active[y] = 1
    return dict(breaking=breaking, breaking_prev=breaking_prev, arising=arising,
                active=active, global_trigger=int(breaking.size + arising.size > 0))


# ----------------------------------------------------------------------------
# Section 3.2.4 "Extracting Topology Change Events": bulk and boundary events
# ----------------------------------------------------------------------------

#: bits of the per-label event flags (bit 0 is the local trigger itself)
EV_ACTIVE, EV_BULK, EV_BOUNDARY, EV_BPOINT_NOW, EV_BPOINT_PAST = 1, 2, 4, 8, 16


def adjacency(E: np.ndarray, K: int) -> list:
    """Neighbour sets of labels 0..K-1 from sorted link keys (both directions)."""
    nb = [set() for _ in range(K)]
    a, b = split_keys(E)
    for x, y in zip(a.tolist(), b.tolist()):
        nb[x].add(y)
        nb[y].add(x)
    return nb


def boundary_point(nb: list, u: int) -> bool:
    """Section 3.2.4: an edge whose two ends share exactly one neighbour is a
    boundary edge (two shared neighbours: bulk edge); both ends of a boundary
    edge are boundary points."""
    return any(len(nb[u] & nb[v]) == 1 for v in nb[u])


def classify_events(E_prev: np.ndarray, E_now: np.ndarray, phi: np.ndarray, inv: np.ndarray,
                    active: np.ndarray) -> np.ndarray:
    """Event flags of the now-labels (Section 3.2.4, "Extracting Topology Change Events").

    The active points are the now-labels with the local trigger set; every one
    is matched (flips only join matched labels), so its past label is
    Phi^-1(a). Readings:

    * eventsCount, counted in each triangulation: c_N(a) = active now
      neighbours of a; c_P(a) = past neighbours q of Phi^-1(a) with Phi(q)
      active (the past configuration seen through the isomorphism).
    * bulk event point: active and, in a single configuration, linked to at
      least three other active points: max(c_N, c_P) >= 3.
    * boundary point of a triangulation: an end of a boundary edge (its two
      ends share exactly one neighbour).
    * boundary event point: active and, in the past or in the now
      triangulation, a boundary point linked to at least one other active
      point that is a boundary point of the same triangulation.

    Returns uint8 flags per now-label: EV_ACTIVE (the local trigger), EV_BULK,
    EV_BOUNDARY, EV_BPOINT_NOW / EV_BPOINT_PAST (the active point is a
    boundary point of that triangulation); inactive labels get 0.
    """
    K_now = inv.shape[0]
    K_prev = phi.shape[0]
    flags = np.zeros(K_now, dtype=np.uint8)
    act = np.asarray(active, dtype=np.uint8) != 0
    if not act.any():
        return flags
    nbN = adjacency(E_now, K_now)
    nbP = adjacency(E_prev, K_prev)

    def active_now(n: int) -> bool:
        return 0 <= n < K_now and bool(act[n])

    def active_past(q: int) -> bool:   # past label q seen through Phi
        return active_now(int(phi[q])) if phi[q] >= 0 else False

    for a in np.flatnonzero(act).tolist():
        ia = int(inv[a])
        f = EV_ACTIVE
        c_now = sum(1 for b in nbN[a] if active_now(b))
        c_past = sum(1 for q in nbP[ia] if active_past(q)) if ia >= 0 else 0
        if max(c_now, c_past) >= 3:
            f |= EV_BULK
        bnow = boundary_point(nbN, a)
        bpast = ia >= 0 and boundary_point(nbP, ia)
        if bnow:
            f |= EV_BPOINT_NOW
        if bpast:
            f |= EV_BPOINT_PAST
        ev_now = bnow and any(active_now(b) and boundary_point(nbN, b) for b in nbN[a])
        ev_past = bpast and any(active_past(q) and boundary_point(nbP, q) for q in nbP[ia])
        if ev_now or ev_past:
            f |= EV_BOUNDARY
        flags[a] = f
    return flags


# ----------------------------------------------------------------------------
# Whole pipeline, one frame after another
# ----------------------------------------------------------------------------

class Detector:
    """Frame-to-frame detector: push fields in order, get every intermediate.

    ``push(F)`` runs threshold -> labels -> Q10 centroids -> Voronoi owners ->
    edge keys on F, then (from the second frame on) the match against the
    previous frame (by overlap, or by centres with ``match="centroid"``), the
    flip lists and, with ``events=True``, the event flags (``active`` carries
    the local trigger in bit 0 and the classes of ``classify_events`` above
    it). The first frame reports no changes.
    """

    def __init__(self, Lx: int, Ly: int, theta: float = 0.5, polarity: int = 1,
                 connectivity: int = 4, workers: int = 1, voronoi: str = "kdtree",
                 events: bool = False, match: str = "overlap", match_radius: int = 0,
                 edge_rule: str = "adj4", walls=(False, False), obstacles=None):
        self.Lx, self.Ly = Lx, Ly
        self.edge_rule = edge_rule
        self.periodic = (not walls[0], not walls[1])
        self.obstacles = None if obstacles is None else np.asarray(obstacles, dtype=bool)
        self.events = events
        self.match = match
        self.match_radius = match_radius
        self.theta, self.polarity = theta, polarity
        self.connectivity = connectivity
        self.workers = workers
        self.voronoi = voronoi
        self.prev = None
        self.frame = 0

    def push(self, F: np.ndarray) -> dict:
        F = np.asarray(F, dtype=np.float32)
        assert F.shape == (self.Ly, self.Lx)
        fg = foreground(F, self.theta, self.polarity)
        if self.obstacles is not None:
            fg &= ~self.obstacles            # an obstacle site is never in a bubble
        per = self.periodic
        labels, K = label_components(fg, self.connectivity, per)
        cq = centroids_q10(labels, K, per)
        if self.voronoi == "brute" or per != (True, True):
            own = owners_bruteforce(cq, self.Lx, self.Ly, periodic=per)
        else:
            own = owners(cq, self.Lx, self.Ly, workers=self.workers)
        if self.obstacles is not None:
            own = np.where(self.obstacles, OBSTACLE, own).astype(np.int32)
        E = vertex_edges(own, cq, per) if self.edge_rule == "vertex" else delaunay_edges(own, cq, per)
        out = dict(frame=self.frame, labels=labels, K=K, centroids=cq, owners=own, edges=E)
        if self.prev is None:
            out.update(phi=np.zeros(0, np.int32), inv=np.full(K, -1, np.int32),
                       breaking=np.zeros(0, np.uint64), breaking_prev=np.zeros(0, np.uint64),
                       arising=np.zeros(0, np.uint64), active=np.zeros(K, np.uint8),
                       global_trigger=0, K_prev=0, n_matched=0)
        else:
            p = self.prev
            if self.match == "centroid":
                phi, inv = match_centroid(p["centroids"], cq, self.Lx, self.Ly, self.match_radius, per)
            else:
                phi, inv = match_overlap(p["labels"], labels, p["K"], K)
            fl = flips(p["edges"], E, phi, inv)
            if self.events:
                fl["active"] = classify_events(p["edges"], E, phi, inv, fl["active"])
            out.update(phi=phi, inv=inv, K_prev=p["K"], n_matched=int((phi >= 0).sum()), **fl)
        self.prev = dict(labels=labels, K=K, edges=E, centroids=cq)
        self.frame += 1
        return out
