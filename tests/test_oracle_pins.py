"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
fixtures under tests/golden/, brute force on tiny inputs (BFS flood fill,
all-centres argmin, an O(n^4) empty-circle Delaunay), closed forms (centroids
of symmetric shapes), invariants (translation covariance, the torus Euler
relation E = 3V of a triangulation) and constructed events (identity frames,
translations, births, deaths, merges, a single T1 flip).
"""
from __future__ import annotations

import os
import random
from collections import deque

import numpy as np
import pytest

import oracle as O
from paper_1607_00908_gb300 import inputs as I
from tests.delaunay_bruteforce import periodic_delaunay

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = 1024


# ----------------------------------------------------------------------------
# helpers independent of the oracle
# ----------------------------------------------------------------------------

def bfs_labels(fg: np.ndarray, connectivity: int = 4) -> np.ndarray:
    """Flood fill in raster order on the torus: ids come out canonical directly."""
    Ly, Lx = fg.shape
    lab = -np.ones((Ly, Lx), dtype=np.int64)
    if connectivity == 4:
        steps = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    else:
        steps = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0)]
    nxt = 0
    for y in range(Ly):
        for x in range(Lx):
            if fg[y, x] and lab[y, x] < 0:
                lab[y, x] = nxt
                dq = deque([(x, y)])
                while dq:
                    cx, cy = dq.popleft()
                    for dx, dy in steps:
                        nx, ny = (cx + dx) % Lx, (cy + dy) % Ly
                        if fg[ny, nx] and lab[ny, nx] < 0:
                            lab[ny, nx] = nxt
                            dq.append((nx, ny))
                nxt += 1
    return lab


def renumber_canonical(lab: np.ndarray) -> np.ndarray:
    """Relabel so ids are ranks of each label's first raster-order site."""
    flat = lab.ravel()
    out = -np.ones_like(flat)
    seen = {}
    for i, v in enumerate(flat.tolist()):
        if v >= 0:
            if v not in seen:
                seen[v] = len(seen)
            out[i] = seen[v]
    return out.reshape(lab.shape)


def read_golden(name):
    sections = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("Lx", "Ly", "K"):
                sections[parts[0]] = int(parts[1])
            elif len(parts) == 1 and not parts[0].lstrip("-").isdigit():
                cur = parts[0]
                sections[cur] = []
            else:
                sections.setdefault(cur, []).append([int(float(p)) for p in parts])
    return sections


# ----------------------------------------------------------------------------
# Section 3.1: labelling
# ----------------------------------------------------------------------------

def test_golden_ccl_centroids():
    g = read_golden("ccl_centroid_6x5.txt")
    F = np.array(g["field"], dtype=np.float32)
    lab, K = O.label_components(O.foreground(F, 0.5))
    assert K == g["K"]
    assert np.array_equal(lab, np.array(g["labels"]))
    cq = O.centroids_q10(lab, K)
    assert np.array_equal(cq, np.array(g["centroids"]))


@pytest.mark.parametrize("conn", [4, 8])
def test_ccl_matches_bfs_on_random_tiny_tori(conn):
    rng = np.random.default_rng(11 + conn)
    for trial in range(300):
        Lx = int(rng.integers(1, 13))
        Ly = int(rng.integers(1, 13))
        p = float(rng.uniform(0.05, 0.95))
        fg = rng.random((Ly, Lx)) < p
        lab, K = O.label_components(fg, conn)
        ref = bfs_labels(fg, conn)
        assert np.array_equal(lab, ref), (trial, Lx, Ly)
        assert K == (ref.max() + 1 if (ref >= 0).any() else 0)


def test_threshold_polarity_and_nan():
    F = np.array([[0.5, 0.50001, np.nan, -1.0, 2.0]], dtype=np.float32)
    assert O.foreground(F, 0.5, +1).tolist() == [[False, True, False, False, True]]
    assert O.foreground(F, 0.5, -1).tolist() == [[False, False, False, True, False]]


def test_ccl_roll_covariance():
    F = I.smoothed_noise(96, 80, 3.0, seed=4)
    lab, K = O.label_components(O.foreground(F))
    for sx, sy in [(1, 0), (0, 1), (17, 33), (79, 95)]:
        Fr = np.roll(np.roll(F, sy, axis=0), sx, axis=1)
        labr, Kr = O.label_components(O.foreground(Fr))
        assert Kr == K
        expect = renumber_canonical(np.roll(np.roll(lab, sy, axis=0), sx, axis=1))
        assert np.array_equal(labr, expect)


def test_ccl_discs_are_components():
    st = I.rsa_discs(192, seed=2, max_consecutive_rejections=20000)
    F = I.raster_discs(st)
    lab, K = O.label_components(O.foreground(F))
    assert K == st.n
    # every disc's raster is exactly one component
    for i in range(st.n):
        one = I.raster_discs(I.DiscState(st.L, st.cx[i:i + 1], st.cy[i:i + 1], st.r[i:i + 1]))
        sites = one > 0.5
        vals = np.unique(lab[sites])
        assert vals.size == 1 and vals[0] >= 0
        assert int((lab == vals[0]).sum()) == int(sites.sum())


# ----------------------------------------------------------------------------
# Section 3.1: centre of mass
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("w,h", [(1, 1), (3, 5), (4, 4), (6, 3), (7, 8)])
def test_centroid_closed_form_rectangles_across_seams(w, h):
    """A w x h block has its centre at x0 + (w-1)/2, y0 + (h-1)/2 exactly."""
    Lx, Ly = 23, 19
    for x0 in (0, 5, Lx - 2, Lx - 1):
        for y0 in (0, 7, Ly - 3):
            F = np.zeros((Ly, Lx), np.float32)
            for dy in range(h):
                for dx in range(w):
                    F[(y0 + dy) % Ly, (x0 + dx) % Lx] = 1.0
            lab, K = O.label_components(O.foreground(F))
            assert K == 1
            cq = O.centroids_q10(lab, K)
            ex = (Q * (2 * x0 + w - 1)) // 2 % (Q * Lx)
            ey = (Q * (2 * y0 + h - 1)) // 2 % (Q * Ly)
            assert tuple(cq[0]) == (ex, ey)


@pytest.mark.parametrize("L", [5, 7, 23])
def test_centroid_closed_form_half_ring_bars(L):
    """A bar of w = ceil(L/2) sites starting at its own first site: every
    displacement 0..w-1 lies inside the minimum-image window, so the centroid
    is the bar's midpoint, in both axes and on odd rings too."""
    w = (L + 1) // 2
    for y0 in range(L):
        F = np.zeros((L, L), np.float32)
        F[y0, 0:w] = 1.0
        lab, K = O.label_components(O.foreground(F))
        cq = O.centroids_q10(lab, K)
        assert tuple(cq[0]) == ((Q * (w - 1)) // 2, Q * y0)
        lab, K = O.label_components(O.foreground(F.T.copy()))
        cq = O.centroids_q10(lab, K)
        assert tuple(cq[0]) == (Q * y0, (Q * (w - 1)) // 2)


def test_centroid_closed_form_discs_on_grid_points():
    """A disc raster centred on an integer or half-integer point is symmetric."""
    L = 40
    for cx, cy in [(10.0, 10.0), (0.0, 0.0), (39.5, 20.5), (0.5, 39.0), (20.5, 0.5)]:
        for r in (2.3, 3.7, 5.0):
            st = I.DiscState(L, np.array([cx]), np.array([cy]), np.array([r]))
            F = I.raster_discs(st)
            lab, K = O.label_components(O.foreground(F))
            assert K == 1
            cq = O.centroids_q10(lab, K)
            assert tuple(cq[0]) == (int(round(Q * cx)) % (Q * L), int(round(Q * cy)) % (Q * L))


def test_centroid_exact_half_rounds_up():
    """A 64 x 32 block with its corner (63, 31) moved to (64, 0): n = 2048,
    Sx = 32 * 2016 - 63 + 64 = 64513 and Sy = 64 * 496 - 31 = 31713 about the
    first site (0, 0), so 1024 Sx / n = 32256.5 and 1024 Sy / n = 15856.5:
    both exact halves, rounded up."""
    fg = np.zeros((80, 160), dtype=bool)
    fg[:32, :64] = True
    fg[31, 63] = False
    fg[0, 64] = True
    lab, K = O.label_components(fg)
    assert K == 1
    assert O.centroids_q10(lab, K).tolist() == [[32257, 15857]]


@pytest.mark.parametrize("axis", [0, 1])
def test_bar_longer_than_half_a_bounded_axis_has_plain_centre(axis):
    """Walls across the bar's axis, sites 1..8 of a 10-site axis: the
    displacements from the first site are plain (0..7), not minimum images
    (which would fold 5, 6, 7 to -5, -4, -3), so the centre is the plain mean
    4.5."""
    fg = np.zeros((10, 4), dtype=bool)
    fg[1:9, 2] = True
    per = (True, False)
    if axis == 0:
        fg, per = fg.T.copy(), (False, True)
    lab, K = O.label_components(fg, 4, per)
    assert K == 1
    c = O.centroids_q10(lab, K, per).tolist()[0]
    assert c[1 - axis] == 2 * Q and c[axis] == Q * 9 // 2


@pytest.mark.parametrize("L,length,wide", [(10, 4, False), (10, 5, True), (10, 10, True),
                                            (11, 5, False), (11, 6, True)])
def test_wide_components_by_extent(L, length, wide):
    """A bar of `length` sites on a periodic ring of L sites is wide exactly
    when 2 * length >= L (the full ring winds around the torus); a bar along
    the other, bounded, axis is never wide, whatever its length."""
    fg = np.zeros((3, L), dtype=bool)
    fg[1, :length] = True
    lab, K = O.label_components(fg)
    assert K == 1 and O.wide_components(lab, K).tolist() == [wide]
    lab, K = O.label_components(fg.T.copy(), 4, (True, False))
    assert K == 1 and O.wide_components(lab, K, (True, False)).tolist() == [False]


def test_wide_components_of_discs_and_a_winding_band():
    """Discs of radius 3 on a 32 x 32 torus are never wide, also across the
    seams; a diagonal band that winds around the torus is."""
    fg = np.zeros((32, 32), dtype=bool)
    y, x = np.mgrid[0:32, 0:32]
    for cx, cy in ((0, 0), (16, 31), (8, 12)):
        dx = (x - cx + 16) % 32 - 16
        dy = (y - cy + 16) % 32 - 16
        fg |= dx * dx + dy * dy <= 9
    lab, K = O.label_components(fg)
    assert K == 3 and not O.wide_components(lab, K).any()
    band = ((x - y) % 32) < 2
    lab, K = O.label_components(band)
    assert K == 1 and O.wide_components(lab, K).tolist() == [True]


def test_wide_bar_centroid_follows_the_first_site():
    """A bar over sites 0..5 of a 10-site ring is wide: from its first site
    x = 0 the displacements are 0, 1, 2, 3, 4 and wrap(5) = -5, so Sx = 5 and
    cx = rdiv(1024 * 5, 6) = 853 (measured from x = 5 it would be 2.5 sites)."""
    fg = np.zeros((3, 10), dtype=bool)
    fg[1, :6] = True
    lab, K = O.label_components(fg)
    assert K == 1 and O.centroids_q10(lab, K).tolist() == [[853, Q]]


def test_centroid_within_half_unit_of_plain_mean():
    """Away from the seams the centroid is the plain mean of coordinates; near a
    seam, rolling the lattice to move the bubble away gives the same answer."""
    F = I.smoothed_noise(64, 72, 2.5, seed=9)
    lab, K = O.label_components(O.foreground(F))
    cq = O.centroids_q10(lab, K)
    Ly, Lx = lab.shape
    for k in range(K):
        ys, xs = np.nonzero(lab == k)
        # roll so that the bubble's first site sits at the lattice centre
        first = int(np.flatnonzero(lab.ravel() == k)[0])
        fy, fx = divmod(first, Lx)
        sx, sy = Lx // 2 - fx, Ly // 2 - fy
        xr = (xs + sx) % Lx
        yr = (ys + sy) % Ly
        if xr.max() - xr.min() >= Lx // 2 or yr.max() - yr.min() >= Ly // 2:
            continue  # too wide for a seam-free view
        mx = Q * (xr.mean() - sx)
        my = Q * (yr.mean() - sy)
        dx = (cq[k, 0] - mx + Q * Lx / 2) % (Q * Lx) - Q * Lx / 2
        dy = (cq[k, 1] - my + Q * Ly / 2) % (Q * Ly) - Q * Ly / 2
        assert abs(dx) <= 0.5 + 1e-9 and abs(dy) <= 0.5 + 1e-9


def _narrow(lab, k):
    """True when bubble k fits in a half-lattice window around its first site."""
    Ly, Lx = lab.shape
    first = int(np.flatnonzero(lab.ravel() == k)[0])
    fy, fx = divmod(first, Lx)
    ys, xs = np.nonzero(lab == k)
    dx = (xs - fx + Lx // 2) % Lx - Lx // 2
    dy = (ys - fy + Ly // 2) % Ly - Ly // 2
    return dx.max() - dx.min() < Lx // 2 - 1 and dy.max() - dy.min() < Ly // 2 - 1 \
        and abs(dx).max() < Lx // 2 - 1 and abs(dy).max() < Ly // 2 - 1


def test_centroid_translation_covariance():
    """Shifting the field by whole sites shifts every narrow bubble's centroid
    by exactly 1024 units per site (bubbles spanning half the lattice or more
    have a root-dependent minimum image and are excluded)."""
    F = I.smoothed_noise(48, 56, 2.0, seed=5)
    lab, K = O.label_components(O.foreground(F))
    cq = O.centroids_q10(lab, K)
    narrow = [k for k in range(K) if _narrow(lab, k)]
    assert len(narrow) >= 5
    for sx, sy in [(3, 0), (0, 11), (29, 47)]:
        labr, Kr = O.label_components(O.foreground(np.roll(np.roll(F, sy, 0), sx, 1)))
        cqr = O.centroids_q10(labr, Kr)
        for k in narrow:
            first = int(np.flatnonzero(lab.ravel() == k)[0])
            y, x = divmod(first, 56)
            kr = labr[(y + sy) % 48, (x + sx) % 56]
            assert tuple(cqr[kr]) == ((cq[k, 0] + Q * sx) % (Q * 56), (cq[k, 1] + Q * sy) % (Q * 48))


# ----------------------------------------------------------------------------
# Section 3.2.1: Voronoi colouring
# ----------------------------------------------------------------------------

def test_golden_voronoi_ring():
    g = read_golden("voronoi_ring_8x1.txt")
    cq = np.array(g["centroids"], dtype=np.int64)
    own = O.owners(cq, g["Lx"], g["Ly"])
    assert own.ravel().tolist() == g["owners"][0]
    E = O.delaunay_edges(own, cq)
    assert [tuple(p) for p in zip(*O.split_keys(E))] == [tuple(g["edges"][0])]


def test_owners_kdtree_matches_bruteforce():
    rng = np.random.default_rng(3)
    for trial in range(60):
        Lx = int(rng.integers(1, 40))
        Ly = int(rng.integers(1, 40))
        K = int(rng.integers(1, 25))
        if trial % 3 == 0:
            # centres on lattice points and half points: many exact ties
            cq = np.stack([rng.integers(0, 2 * Lx, K) * (Q // 2),
                           rng.integers(0, 2 * Ly, K) * (Q // 2)], 1).astype(np.int64)
        else:
            cq = np.stack([rng.integers(0, Q * Lx, K), rng.integers(0, Q * Ly, K)], 1).astype(np.int64)
        a = O.owners(cq, Lx, Ly)
        b = O.owners_bruteforce(cq, Lx, Ly)
        assert np.array_equal(a, b), trial


def test_owner_tie_goes_to_smallest_label():
    # site (4, 4) at (4096, 4096); ids 3 and 7 both at squared distance 2*1024^2
    Lx = Ly = 16
    cq = np.array([[12000, 12000 + 7 * j] for j in range(10)], dtype=np.int64)
    cq[3] = (3072, 3072)
    cq[7] = (5120, 5120)
    own = O.owners(cq, Lx, Ly)
    assert own[4, 4] == 3
    own_b = O.owners_bruteforce(cq, Lx, Ly)
    assert own_b[4, 4] == 3
    # same with the labels swapped: still the smaller one wins
    cq[[3, 7]] = cq[[7, 3]]
    assert O.owners(cq, Lx, Ly)[4, 4] == 3


def test_owners_without_centres_are_minus_one():
    """With no centre (no bubble) no site has an owner, in both the literal
    definition and the k-d tree path."""
    cq = np.zeros((0, 2), dtype=np.int64)
    assert (O.owners_bruteforce(cq, 5, 4) == -1).all() and O.owners_bruteforce(cq, 5, 4).shape == (4, 5)
    assert (O.owners(cq, 5, 4) == -1).all()


def test_first_frame_reports_no_changes():
    """The first frame has no past: no match, no flips, no trigger."""
    F = I.smoothed_noise(48, 48, 2.5, seed=3)
    r = O.Detector(48, 48, voronoi="brute", events=True).push(F)
    assert r["K"] > 0 and r["global_trigger"] == 0 and r["K_prev"] == 0 and r["n_matched"] == 0
    assert r["breaking"].size == r["arising"].size == r["breaking_prev"].size == 0
    assert not r["active"].any() and (r["inv"] == -1).all()


def test_owners_translation_covariance():
    rng = np.random.default_rng(8)
    Lx, Ly, K = 37, 29, 15
    cq = np.stack([rng.integers(0, Q * Lx, K), rng.integers(0, Q * Ly, K)], 1).astype(np.int64)
    own = O.owners(cq, Lx, Ly)
    for sx, sy in [(1, 0), (5, 9), (36, 28)]:
        cs = np.stack([(cq[:, 0] + Q * sx) % (Q * Lx), (cq[:, 1] + Q * sy) % (Q * Ly)], 1)
        assert np.array_equal(O.owners(cs, Lx, Ly), np.roll(np.roll(own, sy, 0), sx, 1))


def test_owners_empty_and_single():
    assert (O.owners(np.zeros((0, 2), np.int64), 5, 4) == -1).all()
    assert (O.owners(np.array([[100, 200]]), 5, 4) == 0).all()
    assert O.delaunay_edges(O.owners(np.zeros((0, 2), np.int64), 5, 4), np.zeros((0, 2))).size == 0


# ----------------------------------------------------------------------------
# Section 3.2.2: edges
# ----------------------------------------------------------------------------

def test_golden_plaquette_incircle():
    rows = read_golden("plaquette_incircle.txt")[None]
    for ax, ay, bx, by, cx, cy, dx, dy, lo, hi in rows:
        cq = np.array([[ax, ay], [bx, by], [cx, cy], [dx, dy]], dtype=np.int64)
        assert O.plaquette_diagonal(0, 1, 2, 3, cq, 64, 64) == (lo, hi)


def test_golden_plaquette_owners():
    g = read_golden("plaquette_owners_10x10.txt")
    own = np.array(g["owners"], dtype=np.int32)
    cq = np.array(g["centroids"], dtype=np.int64)
    E = O.delaunay_edges(own, cq)
    assert [list(p) for p in zip(*[v.tolist() for v in O.split_keys(E)])] == g["edges"]


def _generic_points(rng, L, K, min_sep):
    pts = []
    tries = 0
    while len(pts) < K and tries < 10000:
        tries += 1
        p = (int(rng.integers(0, Q * L)), int(rng.integers(0, Q * L)))
        ok = True
        for q in pts:
            dx = O.wrap(p[0] - q[0], Q * L)
            dy = O.wrap(p[1] - q[1], Q * L)
            if dx * dx + dy * dy < (min_sep * Q) ** 2:
                ok = False
                break
        if ok:
            pts.append(p)
    return pts


def _jittered_triangular(rng, a, m, n, Lx, Ly, jitter):
    pts = []
    for j in range(n):
        for i in range(m):
            x = (i * a + (j % 2) * a / 2 + rng.uniform(-jitter, jitter)) % Lx
            y = (j * Ly / n + rng.uniform(-jitter, jitter)) % Ly
            pts.append((int(x * Q), int(y * Q)))
    return pts


def test_edges_equal_bruteforce_delaunay_on_generic_configurations():
    """Jittered triangular lattices have every dual Voronoi edge several sites
    long. For those (no cocircular quadruple, every dual edge longer than 3
    sites) the digital edge set is exactly the periodic Delaunay
    triangulation, and it satisfies the torus Euler relation E = 3K."""
    rng = np.random.default_rng(21)
    a, m, n = 12, 6, 4
    Lx, Ly = a * m, 42
    K = m * n
    checked = 0
    for trial in range(12):
        pts = _jittered_triangular(rng, a, m, n, Lx, Ly, jitter=1.5)
        edges, tris, margin, dual, _ = periodic_delaunay(pts, Q * Lx, Q * Ly, radius=int(2.5 * a * Q))
        assert len(tris) == 3 * 2 * K          # each of the 2K triangles seen from its 3 vertices
        if margin == 0 or dual < 3 * Q or len(edges) != 3 * K:
            continue
        cq = np.array(pts, dtype=np.int64)
        own = O.owners_bruteforce(cq, Lx, Ly)
        E = O.delaunay_edges(own, cq)
        got = set(zip(*[a_.tolist() for a_ in O.split_keys(E)]))
        assert got == edges, trial
        assert len(E) == 3 * K
        checked += 1
    assert checked >= 5


def test_edges_differ_from_delaunay_only_near_degenerate_quads():
    """On random point sets every Delaunay edge whose dual Voronoi edge is at
    least 2*sqrt(2) sites long is found, and every extra digital link is the
    other diagonal of a quad whose Delaunay diagonal has a short dual edge."""
    rng = np.random.default_rng(22)
    L, K = 48, 14
    for trial in range(8):
        pts = _generic_points(rng, L, K, min_sep=7)
        edges, tris, margin, dual, dual_of = periodic_delaunay(pts, Q * L, Q * L, radius=int(0.8 * L * Q))
        assert len(tris) == 3 * 2 * K
        cq = np.array(pts, dtype=np.int64)
        E = O.delaunay_edges(O.owners_bruteforce(cq, L, L), cq)
        got = set(zip(*[a_.tolist() for a_ in O.split_keys(E)]))
        for e in edges - got:
            assert dual_of[e] < 2 * np.sqrt(2) * Q, (trial, e, dual_of[e] / Q)
        short = [e for e in edges if dual_of[e] < 2 * np.sqrt(2) * Q]
        short_ends = set(x for e in short for x in e)
        for e in got - edges:
            assert e[0] in short_ends and e[1] in short_ends, (trial, e)
        # the digital links still form a triangulation: a missing Delaunay
        # edge is replaced by the other diagonal of its quad
        nb = {}
        for x, y in edges:
            nb.setdefault(x, set()).add(y)
            nb.setdefault(y, set()).add(x)
        for e in edges - got:
            opp = sorted(nb[e[0]] & nb[e[1]])
            if len(opp) == 2:
                assert (opp[0], opp[1]) in got, (trial, e, opp)
        if len(edges) == 3 * K:
            assert len(got) == 3 * K, trial


def test_links_translation_covariance_across_seams():
    """Rolling the owner map by whole sites and moving every centre with it
    leaves the link set unchanged, also where a four-colour plaquette's centres
    straddle a seam (the plaquette test unwraps them around one corner).
    Centres near a square lattice make four-cell junctions, so four-colour
    plaquettes are common."""
    rng = np.random.default_rng(31)
    a, m = 8, 5
    L = a * m
    seen_four = 0
    for trial in range(4):
        pts = [(int((i * a + a / 2 + rng.uniform(-0.3, 0.3)) * Q), int((j * a + a / 2 + rng.uniform(-0.3, 0.3)) * Q))
               for j in range(m) for i in range(m)]
        cq = np.array(pts, dtype=np.int64)
        own = O.owners_bruteforce(cq, L, L)
        A = own
        B = np.roll(A, -1, 1)
        C = np.roll(B, -1, 0)
        D = np.roll(A, -1, 0)
        seen_four += int(((A != B) & (A != C) & (A != D) & (B != C) & (B != D) & (C != D)).sum())
        E = O.delaunay_edges(own, cq)
        for _ in range(6):
            sx, sy = (int(v) for v in rng.integers(0, L, size=2))
            own2 = np.roll(np.roll(own, sy, axis=0), sx, axis=1)
            cq2 = (cq + Q * np.array([sx, sy], dtype=np.int64)) % (Q * L)
            assert O.delaunay_edges(own2, cq2).tolist() == E.tolist(), (trial, sx, sy)
    assert seen_four >= 10


def test_every_cell_connected_on_generic_configurations():
    rng = np.random.default_rng(5)
    L, K = 40, 12
    for _ in range(10):
        pts = _generic_points(rng, L, K, min_sep=8)
        cq = np.array(pts, dtype=np.int64)
        own = O.owners_bruteforce(cq, L, L)
        for k in range(len(pts)):
            lab, n = O.label_components(own == k, connectivity=8)
            assert n == 1


# ----------------------------------------------------------------------------
# Sections 3.2.3-3.2.4: match and flips
# ----------------------------------------------------------------------------

def _disc_field(L, pts, r):
    st = I.DiscState(L, np.array([p[0] for p in pts], float), np.array([p[1] for p in pts], float),
                     np.full(len(pts), r, float))
    return I.raster_discs(st)


def test_identity_frame_has_identity_match_and_no_flips():
    F = I.smoothed_noise(64, 64, 3.0, seed=1)
    d = O.Detector(64, 64, voronoi="brute")
    d.push(F)
    r = d.push(F.copy())
    assert np.array_equal(r["phi"], np.arange(r["K"]))
    assert r["breaking"].size == 0 and r["arising"].size == 0 and r["global_trigger"] == 0


def test_integer_translation_is_a_bijection_with_no_flips():
    """Droplets (radius >= 4) moved by a whole-site shift smaller than their size
    overlap their own past selves most: Phi is a bijection, and the Voronoi
    diagram moves rigidly, so no link breaks or arises."""
    st = I.rsa_discs(96, seed=6, rmin=4.0, rmax=6.0, max_consecutive_rejections=5000)
    F = I.raster_discs(st)
    Ly, Lx = F.shape
    d = O.Detector(Lx, Ly, voronoi="brute")
    r0 = d.push(F)
    sx, sy = 2, 1
    r1 = d.push(np.roll(np.roll(F, sy, 0), sx, 1))
    assert r0["K"] == st.n
    assert r1["n_matched"] == r0["K"] == r1["K"]
    # Phi(p) is the now-label found at p's first site shifted by (sx, sy)
    lab0 = r0["labels"]
    for p in range(r0["K"]):
        first = int(np.flatnonzero(lab0.ravel() == p)[0])
        y, x = divmod(first, Lx)
        assert r1["phi"][p] == r1["labels"][(y + sy) % Ly, (x + sx) % Lx]
    assert r1["breaking"].size == 0 and r1["arising"].size == 0


def _disc_label_map(lab, pts):
    """label -> disc index, by the label at each disc's centre site."""
    m = {}
    for i, (x, y) in enumerate(pts):
        m[int(lab[int(y), int(x)])] = i
    return m


def test_single_t1_flip_matches_bruteforce_delaunay_difference():
    """A T1 event built by hand: in a jittered triangular packing pick a
    Delaunay edge (i, k), and squeeze its two opposite droplets j, l toward each
    other past the cocircular point. Where the brute-force triangulation of the
    centroids of both frames changes by exactly that one flip (and the digital
    edge sets equal it in both frames), the oracle must report exactly one
    breaking link {i, k}, one arising link {j, l}, and four active labels (a
    bulk T1 conserves coordination)."""
    rng = np.random.default_rng(7)
    a, m, n = 12, 6, 4
    Lx, Ly = a * m, 42
    K = m * n
    r = 3.0
    found = 0
    for trial in range(40):
        base = _jittered_triangular(rng, a, m, n, Lx, Ly, jitter=0.8)
        pts0 = [(p[0] // Q + 0.5, p[1] // Q + 0.5) for p in base]
        cq0 = [(int(Q * x), int(Q * y)) for x, y in pts0]
        e_base, _, _, _, _ = periodic_delaunay(cq0, Q * Lx, Q * Ly, 2 * a * Q)
        i, k = sorted(e_base)[int(rng.integers(len(e_base)))]
        nb = {}
        for x, y in e_base:
            nb.setdefault(x, set()).add(y)
            nb.setdefault(y, set()).add(x)
        opp = sorted(nb[i] & nb[k])
        if len(opp) != 2:
            continue
        j, l = opp
        vx = float(O.wrap(int(Q * (pts0[l][0] - pts0[j][0])), Q * Lx)) / Q
        vy = float(O.wrap(int(Q * (pts0[l][1] - pts0[j][1])), Q * Ly)) / Q
        dist = np.hypot(vx, vy)
        s = rng.uniform(4.5, 5.5)
        pts1 = list(pts0)
        pts1[j] = ((int(np.floor(pts0[j][0] + s * vx / dist)) % Lx) + 0.5,
                   (int(np.floor(pts0[j][1] + s * vy / dist)) % Ly) + 0.5)
        pts1[l] = ((int(np.floor(pts0[l][0] - s * vx / dist)) % Lx) + 0.5,
                   (int(np.floor(pts0[l][1] - s * vy / dist)) % Ly) + 0.5)
        st0 = I.DiscState(Lx, np.array([p[0] for p in pts0]), np.array([p[1] for p in pts0]), np.full(K, r))
        st1 = I.DiscState(Lx, np.array([p[0] for p in pts1]), np.array([p[1] for p in pts1]), np.full(K, r))
        d = O.Detector(Lx, Ly, voronoi="brute", events=True)
        ra = d.push(_raster_rect(st0, Lx, Ly))
        rb = d.push(_raster_rect(st1, Lx, Ly))
        if ra["K"] != K or rb["K"] != K or rb["n_matched"] != K:
            continue
        m0 = _disc_label_map(ra["labels"], pts0)
        m1 = _disc_label_map(rb["labels"], pts1)
        if len(m0) != K or len(m1) != K:
            continue
        e0, t0, g0, _, _ = periodic_delaunay([tuple(c) for c in ra["centroids"].tolist()], Q * Lx, Q * Ly, 2 * a * Q)
        e1, t1, g1, _, _ = periodic_delaunay([tuple(c) for c in rb["centroids"].tolist()], Q * Lx, Q * Ly, 2 * a * Q)
        if len(t0) != 6 * K or len(t1) != 6 * K or min(g0, g1) == 0:
            continue
        got0 = set(zip(*[v.tolist() for v in O.split_keys(ra["edges"])]))
        got1 = set(zip(*[v.tolist() for v in O.split_keys(rb["edges"])]))
        if got0 != e0 or got1 != e1:
            continue
        s0 = {tuple(sorted((m0[x], m0[y]))) for x, y in e0}
        s1 = {tuple(sorted((m1[x], m1[y]))) for x, y in e1}
        if s0 - s1 != {(min(i, k), max(i, k))} or s1 - s0 != {(min(j, l), max(j, l))}:
            continue
        brk = {tuple(sorted((m1[x], m1[y]))) for x, y in zip(*[v.tolist() for v in O.split_keys(rb["breaking"])])}
        ari = {tuple(sorted((m1[x], m1[y]))) for x, y in zip(*[v.tolist() for v in O.split_keys(rb["arising"])])}
        assert brk == s0 - s1 and ari == s1 - s0
        assert int((rb["active"] & O.EV_ACTIVE).sum()) == 4
        # a bulk T1 on the torus: the four active labels are bulk event points
        # (each linked to three active labels in one triangulation), and no
        # edge of a periodic triangulation is a boundary edge
        act = np.flatnonzero(rb["active"])
        assert act.size == 4
        assert all(int(rb["active"][x]) == O.EV_ACTIVE | O.EV_BULK for x in act.tolist())
        prev = {tuple(sorted((m0[x], m0[y]))) for x, y in zip(*[v.tolist() for v in O.split_keys(rb["breaking_prev"])])}
        assert prev == s0 - s1
        found += 1
        if found >= 2:
            break
    assert found >= 1


def _raster_rect(st, Lx, Ly):
    """Disc raster on an Lx x Ly torus (the generator's raster is square-only)."""
    F = np.zeros((Ly, Lx), np.float32)
    for cx, cy, r in zip(st.cx, st.cy, st.r):
        R = int(np.ceil(r)) + 1
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                x = int(np.floor(cx)) + dx
                y = int(np.floor(cy)) + dy
                if (x - cx) ** 2 + (y - cy) ** 2 < r * r:
                    F[y % Ly, x % Lx] = 1.0
    return F


def test_birth_and_death_are_excluded():
    L = 64
    rng = np.random.default_rng(4)
    pts = [(p[0] // Q + 0.5, p[1] // Q + 0.5) for p in _generic_points(rng, L, 12, min_sep=12)]
    extra = ((pts[0][0] + 6.0) % L, (pts[0][1] + 6.0) % L)
    F0 = _disc_field(L, pts, 2.2)
    F1 = _disc_field(L, pts + [extra], 2.2)
    for frames, kind in (((F0, F1), "birth"), ((F1, F0), "death")):
        d = O.Detector(L, L, voronoi="brute")
        a = d.push(frames[0])
        b = d.push(frames[1])
        if kind == "birth":
            new = int(b["labels"][int(extra[1]), int(extra[0])])
            assert b["inv"][new] == -1
            ends = set(O.split_keys(b["breaking"])[0].tolist() + O.split_keys(b["breaking"])[1].tolist()
                       + O.split_keys(b["arising"])[0].tolist() + O.split_keys(b["arising"])[1].tolist())
            assert new not in ends
            assert b["n_matched"] == a["K"]
        else:
            gone = int(a["labels"][int(extra[1]), int(extra[0])])
            assert b["inv"].tolist().count(-1) == 0
            assert a["K"] - b["n_matched"] == 1
            assert gone not in [p for p in range(a["K"]) if b["phi"][p] >= 0]


def test_merge_keeps_only_the_mutual_best():
    L = 48
    F0 = np.zeros((L, L), np.float32)
    F0[10:14, 10:16] = 1.0      # p0: 24 sites
    F0[10:14, 17:20] = 1.0      # p1: 12 sites
    F1 = F0.copy()
    F1[10:14, 16] = 1.0          # bridge: one bubble
    d = O.Detector(L, L, voronoi="brute")
    d.push(F0)
    b = d.push(F1)
    assert b["K"] == 1 and b["K_prev"] == 2
    assert b["phi"].tolist() == [0, -1]


def test_overlap_tie_goes_to_smallest_label():
    # two past labels tie for one now label: the smaller past label wins
    lab_prev = np.array([[0, 0, 1, 1]], dtype=np.int32)
    lab_now = np.array([[0, 0, 0, 0]], dtype=np.int32)
    phi, inv = O.match_overlap(lab_prev, lab_now, 2, 1)
    assert phi.tolist() == [0, -1] and inv.tolist() == [0]
    # one past label splits evenly into two now labels: the smaller now label wins
    phi, inv = O.match_overlap(lab_now, lab_prev, 1, 2)
    assert phi.tolist() == [0] and inv.tolist() == [0, -1]
    # a strictly larger overlap beats a smaller label
    phi, inv = O.match_overlap(np.array([[0, 0, 0, 0, 0]], np.int32),
                               np.array([[0, 1, 1, 1, -1]], np.int32), 1, 2)
    assert phi.tolist() == [1] and inv.tolist() == [-1, 0]


# ----------------------------------------------------------------------------
# Section 3.2.4 "Extracting Topology Change Events": hand-built triangulations
# whose event classes follow from the definitions by counting
# ----------------------------------------------------------------------------

def _keys(pairs):
    return np.sort(O.make_keys([p[0] for p in pairs], [p[1] for p in pairs])) if pairs else np.zeros(0, np.uint64)


def _events(past, now, K):
    phi = np.arange(K, dtype=np.int32)
    inv = np.arange(K, dtype=np.int32)
    fl = O.flips(_keys(past), _keys(now), phi, inv)
    return fl, O.classify_events(_keys(past), _keys(now), phi, inv, fl["active"])


def test_breaking_prev_stays_aligned_with_breaking():
    """Phi reverses four labels: past links 0-1 and 2-3 become 3-2 and 1-0 and
    both break. Sorted by now-key the breaking list is (0,1), (2,3); the past
    keys follow it pair by pair: (2,3), (0,1)."""
    phi = np.array([3, 2, 1, 0], dtype=np.int32)
    inv = np.array([3, 2, 1, 0], dtype=np.int32)
    fl = O.flips(O.make_keys([0, 2], [1, 3]), np.zeros(0, np.uint64), phi, inv)
    assert fl["breaking"].tolist() == O.make_keys([0, 2], [1, 3]).tolist()
    assert fl["breaking_prev"].tolist() == O.make_keys([2, 0], [3, 1]).tolist()


def test_centroid_match_with_walls_in_both_directions():
    """Past centre at x = 0.25 of a 10-site axis, now centres at 9.75 and 1.5,
    radius 2. On the torus 9.75 is 0.5 away through the seam and matches;
    with walls only the plain distances count, in both directions of the
    mutual test, and 1.5 (1.25 away) matches."""
    p = np.array([[Q // 4, Q]], dtype=np.int64)
    n = np.array([[Q * 9 + 3 * Q // 4, Q], [3 * Q // 2, Q]], dtype=np.int64)
    assert O.match_centroid(p, n, 10, 3, radius=2)[0].tolist() == [0]
    assert O.match_centroid(p, n, 10, 3, radius=2, periodic=(False, True))[0].tolist() == [1]


def test_detector_passes_its_options():
    """The whole-frame detector applies its options: 8-connectivity joins two
    diagonal sites, polarity -1 takes the sites below the threshold, and the
    centre match uses the radius it is given."""
    F = np.zeros((8, 8), dtype=np.float32)
    F[2, 2] = F[3, 3] = 1.0
    assert O.Detector(8, 8).push(F)["K"] == 2
    assert O.Detector(8, 8, connectivity=8).push(F)["K"] == 1
    assert O.Detector(8, 8, polarity=-1).push(F)["K"] == 1          # the background, one piece
    G = np.zeros((32, 32), dtype=np.float32)
    G[10:13, 10:13] = 1.0
    H = np.roll(G, 3, axis=1)                                        # the block moves 3 sites
    for radius, want in ((4, [0]), (2, [-1])):
        d = O.Detector(32, 32, match="centroid", match_radius=radius)
        d.push(G)
        assert d.push(H)["phi"].tolist() == want, radius


def test_centroid_match_radius_is_inclusive():
    """Centres exactly 3 sites apart match within radius 3 and not within 2."""
    p = np.array([[Q * 2, Q * 2]], dtype=np.int64)
    n = np.array([[Q * 5, Q * 2]], dtype=np.int64)
    assert O.match_centroid(p, n, 16, 16, radius=3)[0].tolist() == [0]
    assert O.match_centroid(p, n, 16, 16, radius=2)[0].tolist() == [-1]


def test_global_trigger_with_one_kind_of_flip():
    """A link that only arises (or only breaks) between matched labels still
    sets the global trigger and the local trigger of its ends."""
    ident = np.arange(3, dtype=np.int32)
    fl = O.flips(O.make_keys([0], [1]), O.make_keys([0, 1], [1, 2]), ident, ident)
    assert fl["breaking"].size == 0 and fl["arising"].tolist() == O.make_keys([1], [2]).tolist()
    assert fl["global_trigger"] == 1 and fl["active"].tolist() == [0, 1, 1]
    fl = O.flips(O.make_keys([0, 1], [1, 2]), O.make_keys([0], [1]), ident, ident)
    assert fl["arising"].size == 0 and fl["breaking"].tolist() == O.make_keys([1], [2]).tolist()
    assert fl["global_trigger"] == 1 and fl["active"].tolist() == [0, 1, 1]


def _wheel(missing=()):
    """Hub 0 joined to rim 1..6, rim joined in a cycle: each rim link's ends
    share only the hub (boundary links, so the rim labels are boundary points);
    each spoke's ends share two rim labels (the hub is not a boundary point)."""
    pairs = [(0, i) for i in range(1, 7)] + [(i, i % 6 + 1) for i in range(1, 7)]
    pairs = [p for p in pairs if p not in missing]
    return O.make_keys([p[0] for p in pairs], [p[1] for p in pairs])


def test_event_classes_on_a_wheel_by_counting():
    """Same wheel before and after, identity match, active labels given:
    {hub, 1}: 1 is a boundary point whose only active neighbour (the hub) is
    not one, and the hub is not a boundary point -- no boundary event, and
    one active neighbour each -- no bulk event. {hub, 1, 2}: 1 and 2 are
    active boundary points linked to each other -- boundary events; every
    active label has two active neighbours -- still no bulk event (three are
    needed)."""
    E = _wheel()
    ident = np.arange(7, dtype=np.int32)
    bp = O.EV_BPOINT_NOW | O.EV_BPOINT_PAST
    act = np.zeros(7, np.uint8)
    act[[0, 1]] = 1
    f = O.classify_events(E, E, ident, ident, act)
    assert f.tolist() == [O.EV_ACTIVE, O.EV_ACTIVE | bp, 0, 0, 0, 0, 0]
    act[2] = 1
    f = O.classify_events(E, E, ident, ident, act)
    be = O.EV_ACTIVE | bp | O.EV_BOUNDARY
    assert f.tolist() == [O.EV_ACTIVE, be, be, 0, 0, 0, 0]


def test_event_classes_follow_a_relabelling_of_the_now_frame():
    """The wheel before and after, the now labels permuted by pi(i) = 6 - i
    (Phi = pi): the flags of now label pi(i) are those label i gets under the
    identity. The past neighbours are seen through Phi, so the hub (now 6)
    still has two active past neighbours (pi(1) = 5 and pi(2) = 4), not
    three."""
    E = _wheel()
    pi = np.array([6 - i for i in range(7)], dtype=np.int32)
    a, b = O.split_keys(E)
    E_now = O.make_keys(pi[a], pi[b])
    ident = np.arange(7, dtype=np.int32)
    act = np.zeros(7, np.uint8)
    act[[0, 1, 2]] = 1
    want = O.classify_events(E, E, ident, ident, act)
    act_pi = np.zeros(7, np.uint8)
    act_pi[pi[[0, 1, 2]]] = 1
    inv = np.argsort(pi).astype(np.int32)
    got = O.classify_events(E, E_now, pi, inv, act_pi)
    assert got[pi].tolist() == want.tolist()
    # no links now: a boundary event can only come from the past wheel, where
    # rim labels 1 and 2 are linked boundary points, active as pi(1), pi(2)
    act_pi[:] = 0
    act_pi[pi[[1, 2]]] = 1
    got = O.classify_events(E, np.zeros(0, np.uint64), pi, inv, act_pi)
    be = O.EV_ACTIVE | O.EV_BPOINT_PAST | O.EV_BOUNDARY
    assert got.tolist() == [0, 0, 0, 0, be, be, 0]


def test_bulk_event_needs_three_in_one_triangulation():
    """Past wheel without the spoke 0-2, now the whole wheel, active {hub, 1, 2}:
    the hub has two active neighbours now and one in the past, label 2 two now
    and one in the past. Three in the two triangulations together, but never
    three in one: no bulk event."""
    ident = np.arange(7, dtype=np.int32)
    act = np.zeros(7, np.uint8)
    act[[0, 1, 2]] = 1
    f = O.classify_events(_wheel(missing=((0, 2),)), _wheel(), ident, ident, act)
    assert not any(int(v) & O.EV_BULK for v in f)


def test_events_boundary_link_breaking():
    """Two triangles (0,1,2), (1,2,3) sharing the bulk edge {1,2}; the boundary
    edge {0,1} (its ends share only label 2) breaks. Labels 0 and 1 are active,
    each linked to one other active label: boundary event points, not bulk.
    In the past both are boundary points; now 1 is still a boundary point
    (edge {1,2} shares only 3), 0 is not (its one edge {0,2} shares nothing)."""
    past = [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)]
    now = [(0, 2), (1, 2), (1, 3), (2, 3)]
    fl, ev = _events(past, now, 4)
    assert fl["breaking"].tolist() == O.make_keys([0], [1]).tolist() and fl["arising"].size == 0
    E = O
    assert ev.tolist() == [E.EV_ACTIVE | E.EV_BOUNDARY | E.EV_BPOINT_PAST,
                           E.EV_ACTIVE | E.EV_BOUNDARY | E.EV_BPOINT_PAST | E.EV_BPOINT_NOW, 0, 0]


def test_events_isolated_rhombus_is_bulk_and_boundary():
    """A lone rhombus A=0, B=1, C=2, D=3 whose diagonal turns from {0,2} to
    {1,3}: every label is linked to the three others in one triangulation
    (bulk), and the rim edges share one label (boundary points linked to
    active boundary points) -- a point in a bulk and a boundary event at once."""
    past = [(0, 1), (1, 2), (2, 3), (0, 3), (0, 2)]
    now = [(0, 1), (1, 2), (2, 3), (0, 3), (1, 3)]
    _, ev = _events(past, now, 4)
    allf = O.EV_ACTIVE | O.EV_BULK | O.EV_BOUNDARY | O.EV_BPOINT_PAST | O.EV_BPOINT_NOW
    assert ev.tolist() == [allf] * 4


def test_events_t1_inside_a_closed_patch_is_bulk_only():
    """The rhombus 0-1-2-3 with its diagonal turning from {0,2} to {1,3},
    closed by two apexes 4 and 5 linked to all four: every link shares at least
    two labels in both frames, so there is no boundary edge and the four
    active labels are bulk event points only."""
    rim = [(0, 1), (1, 2), (2, 3), (0, 3)]
    caps = [(4, 0), (4, 1), (4, 2), (4, 3), (5, 0), (5, 1), (5, 2), (5, 3)]
    past = rim + caps + [(0, 2)]
    now = rim + caps + [(1, 3)]
    # sanity of the construction: label pairs that are linked share >= 2 labels
    for E in (past, now):
        nb = O.adjacency(_keys(E), 6)
        assert all(len(nb[u] & nb[v]) >= 2 for u, v in E)
    _, ev = _events(past, now, 6)
    assert ev.tolist() == [O.EV_ACTIVE | O.EV_BULK] * 4 + [0, 0]


def test_events_identity_and_unmatched():
    """No flip: no flags. An unmatched past label never counts as an active
    neighbour (it has no now label)."""
    past = [(0, 1), (1, 2), (0, 2)]
    _, ev = _events(past, past, 3)
    assert not ev.any()
    # past label 2 unmatched: the now frame has labels 0, 1 only
    phi = np.array([0, 1, -1], np.int32)
    inv = np.array([0, 1], np.int32)
    fl = O.flips(_keys(past), _keys([]), phi, inv)
    ev = O.classify_events(_keys(past), _keys([]), phi, inv, fl["active"])
    assert fl["breaking"].tolist() == O.make_keys([0], [1]).tolist()
    # 0 and 1: one active neighbour each (2 is unmatched), past edge {0,1}
    # shares label 2 only -> boundary points linked to each other
    assert ev.tolist() == [O.EV_ACTIVE | O.EV_BOUNDARY | O.EV_BPOINT_PAST] * 2


# ----------------------------------------------------------------------------
# Section 3.2.3, centre comparison (match_centroid): cases whose Phi follows
# from the definition by hand
# ----------------------------------------------------------------------------

def _q(pts):
    return np.array([[int(Q * x), int(Q * y)] for x, y in pts], dtype=np.int64).reshape(-1, 2)


def test_centroid_match_permuted_translation():
    """Centres moved by a small common shift and relabelled: Phi inverts the
    relabelling (every centre's nearest is its own image, mutually); a shift
    beyond the radius leaves every label unmatched."""
    rng = np.random.default_rng(3)
    L = 200
    g = np.array([(20 * i + 5, 20 * j + 7) for i in range(10) for j in range(10)], dtype=float)
    prev = _q(g)
    perm = rng.permutation(len(g))
    moved = (g + np.array([2.25, -1.5])) % L
    now = _q(moved[perm])
    phi, inv = O.match_centroid(prev, now, L, L, radius=4)
    want = np.empty(len(g), dtype=np.int64)
    want[perm] = np.arange(len(g))
    assert phi.tolist() == want.tolist()
    assert inv.tolist() == perm.tolist()
    phi, inv = O.match_centroid(prev, now, L, L, radius=2)
    assert (phi == -1).all() and (inv == -1).all()


def test_centroid_match_ties_mutuality_and_seam():
    """(a) a past centre midway between two now centres takes the smaller
    label; (b) two past centres near one now centre: only the nearer is
    matched (mutual choice), the other stays unmatched; (c) centres on both
    sides of the periodic seam are 1 site apart, not L - 1."""
    L = 64
    prev = _q([(10, 10)])
    now = _q([(12, 10), (8, 10)])
    phi, inv = O.match_centroid(prev, now, L, L, radius=3)
    assert phi.tolist() == [0] and inv.tolist() == [0, -1]
    prev = _q([(20, 20), (23, 20)])
    now = _q([(21, 20)])
    phi, inv = O.match_centroid(prev, now, L, L, radius=5)
    assert phi.tolist() == [0, -1] and inv.tolist() == [0]
    prev = _q([(0.25, 30), (40, 40)])
    now = _q([(63.5, 30.5), (40, 40)])
    phi, inv = O.match_centroid(prev, now, L, L, radius=1)
    assert phi.tolist() == [0, 1] and inv.tolist() == [0, 1]


def test_centroid_match_equals_bruteforce_loops():
    """The chunked numpy search equals a plain double loop on random centres."""
    rng = np.random.default_rng(11)
    Lx, Ly = 50, 37
    prev = rng.integers(0, [Q * Lx, Q * Ly], size=(40, 2))
    now = (prev[rng.permutation(40)[:33]] + rng.integers(-3 * Q, 3 * Q, size=(33, 2))) % [Q * Lx, Q * Ly]
    R = 4
    phi, inv = O.match_centroid(prev, now, Lx, Ly, radius=R)

    def nearest(q, c):
        best, bd = -1, (Q * R) ** 2
        for j, (x, y) in enumerate(c.tolist()):
            dx = O.wrap(x - int(q[0]), Q * Lx)
            dy = O.wrap(y - int(q[1]), Q * Ly)
            d = dx * dx + dy * dy
            if d < bd or (d == bd and (best < 0 or j < best)):
                best, bd = j, d
        return best

    bn = [nearest(p, now) for p in prev]
    bp = [nearest(n, prev) for n in now]
    want = [bn[p] if bn[p] >= 0 and bp[bn[p]] == p else -1 for p in range(40)]
    assert phi.tolist() == want
    assert sorted(i for i in inv.tolist() if i >= 0) == sorted(p for p in range(40) if want[p] >= 0)


# ----------------------------------------------------------------------------
# Section 3.2.2, the frame rule (vertex_edges, an option; its figures are
# lost, so it is pinned to geometry): hand-counted cases, the periodic
# Delaunay triangulation, pathological colourings and ties
# ----------------------------------------------------------------------------

def test_frame_gaps_and_vertex_links_at_a_three_cell_junction():
    """4 x 4 torus: cell 0 = {x<2, y<2}, cell 1 = {x>=2, y<2}, cell 2 = {y>=2}.
    Frame of (1,1), counter-clockwise from +x: 1,2,2,2,0,0,0,1 -> 3 colour
    changes (a vertex site); frame of (0,0): 0,0,0,1,1,2,2,2 -> 3. At (1,1)
    the +x neighbour (colour 1) passes C(spy)=2 != C(smypx)=1 and the +y
    neighbour (colour 2) passes C(smx)=0 != C(spxpy)=2; at (2,1) the +y
    neighbour (colour 2) passes C(smx)=0 != C(spxpy)=2: the three cells are
    linked pairwise."""
    own = np.array([[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 2, 2], [2, 2, 2, 2]], dtype=np.int32)
    gaps = O.frame_gaps(own)
    assert int(gaps[1, 1]) == 3 and int(gaps[0, 0]) == 3
    cq = np.array([[512, 512], [Q * 2 + 512, 512], [Q + 512, Q * 2 + 512]], dtype=np.int64)
    E = O.vertex_edges(own, cq)
    assert E.tolist() == O.make_keys([0, 0, 1], [1, 2, 2]).tolist()


def test_inner_frame_point_takes_its_exact_voronoi_colour():
    """The fifth second-neighbour condition of Section 3.2.2 reads C(a_k), the
    colour of an inner-frame point, which is a point of the stencil like any
    other: its colour is the Voronoi colour of the point, i.e. the nearest
    centre over all centres. Hand-built 16 x 16 box with walls on both axes,
    so that the four cells meet only once (1/1024-site units):
    centres A, B, C, D sit 0.1 site inside the corners (8,8), (9,8), (9,9),
    (8,9) of one plaquette and E exactly at its centre p = (8.5, 8.5).
    Squared distances to the corner site (8,8): A 2*110^2 = 24,200, E
    2*512^2 = 524,288, so every corner site (and every other site, each at
    least 512*sqrt(2) from E) is owned by one of A-D: E owns no site. Its own
    point p is E's (distance 0). Frame of (8,8), counter-clockwise from +x:
    B C D D A A A B -> 4 colour changes, a vertex site; the diagonal A-C
    passes conditions 1-4 there (C != A, C(spy) = D != C(smypx) = B,
    D != B), and condition 5 reads C(p) = E, neither A nor C: no link. The
    same holds for the diagonal B-D (read at (9,8) and (8,9)) and for A-C read
    from (9,9). A reading that colours p only among the four corner colours
    would give it A (2*402^2 = 323,208 against 2*412^2 = 339,488 for B, C, D)
    and link A-C. The four sides are first-neighbour links, and the four
    sites of the plaquette are the only vertex sites."""
    A, B, C, D, E = 0, 1, 2, 3, 4
    box = (False, False)
    cq = np.array([[8302, 8302], [9116, 8292], [9116, 9116], [8292, 9116], [8704, 8704]], dtype=np.int64)
    own = O.owners_bruteforce(cq, 16, 16, periodic=box)
    assert not (own == E).any()
    assert [int(own[8, 8]), int(own[8, 9]), int(own[9, 9]), int(own[9, 8])] == [A, B, C, D]
    gaps = O.frame_gaps(own, box)
    assert int(gaps[8, 8]) == 4
    assert np.argwhere(gaps >= 3).tolist() == [[8, 8], [8, 9], [9, 8], [9, 9]]
    assert O.owners_at_points(cq, 16, 16, [8704], [8704], box).tolist() == [E]
    keys = O.vertex_edges(own, cq, box)
    assert keys.tolist() == np.sort(O.make_keys([A, B, C, A], [B, C, D, D])).tolist()


def test_points_take_the_owner_of_the_bruteforce_definition():
    """owners_at_points at lattice sites equals the brute-force owners, and at
    half-site points it equals a direct argmin written out for three centres
    with a tie (ties go to the smaller label)."""
    rng = np.random.default_rng(5)
    cq = np.stack([rng.integers(0, Q * 40, 30), rng.integers(0, Q * 24, 30)], axis=1)
    own = O.owners_bruteforce(cq, 40, 24)
    y, x = np.divmod(np.arange(40 * 24), 40)
    assert np.array_equal(O.owners_at_points(cq, 40, 24, Q * x, Q * y), own.ravel())
    # (Q/2, Q/2) is equidistant from (0, Q) and (Q, 0) and farther from (3Q, 3Q)
    cq3 = np.array([[3 * Q, 3 * Q], [Q, 0], [0, Q]], dtype=np.int64)
    assert O.owners_at_points(cq3, 8, 8, [Q // 2], [Q // 2]).tolist() == [1]
    # across the seam: (7.5 Q, 0) is nearer to (0, 0) than to (6 Q, 0) on an 8-site ring
    cq2 = np.array([[6 * Q, 0], [0, 0]], dtype=np.int64)
    assert O.owners_at_points(cq2, 8, 8, [7 * Q + Q // 2], [0]).tolist() == [1]
    assert O.owners_at_points(cq2, 8, 8, [7 * Q + Q // 2], [0], periodic=(False, True)).tolist() == [0]


def test_vertex_rule_sees_no_vertex_between_two_stripes():
    """Two stripes on a torus: every frame changes colour twice at most, so no
    site is a vertex and the frame rule reads no link."""
    own = np.zeros((6, 5), dtype=np.int32)
    own[3:] = 1
    assert int(O.frame_gaps(own).max()) == 2
    cq = np.array([[Q * 2, Q], [Q * 2, Q * 4]], dtype=np.int64)
    assert O.vertex_edges(own, cq).size == 0


def test_vertex_rule_equals_bruteforce_delaunay_on_generic_configurations():
    """Every Voronoi vertex of a generic point set is a site whose frame
    changes colour three times, so the frame rule reads each Delaunay
    triangle there. On jittered triangular lattices (no cocircular
    quadruple, every dual edge longer than 3 sites) its links are exactly the
    periodic Delaunay triangulation found by empty-circle brute force."""
    rng = np.random.default_rng(21)
    a, m, n = 12, 6, 4
    Lx, Ly = a * m, 42
    K = m * n
    checked = 0
    for trial in range(12):
        pts = _jittered_triangular(rng, a, m, n, Lx, Ly, jitter=1.5)
        edges, tris, margin, dual, _ = periodic_delaunay(pts, Q * Lx, Q * Ly, radius=int(2.5 * a * Q))
        if margin == 0 or dual < 3 * Q or len(edges) != 3 * K:
            continue
        cq = np.array(pts, dtype=np.int64)
        E = O.vertex_edges(O.owners_bruteforce(cq, Lx, Ly), cq)
        got = set(zip(*[a_.tolist() for a_ in O.split_keys(E)]))
        assert got == edges, trial
        checked += 1
    assert checked >= 5


def test_vertex_rule_differs_from_delaunay_only_at_near_degenerate_quads():
    """On random point sets the frame rule finds every Delaunay edge whose
    dual Voronoi edge is at least one site long; a missed edge is replaced by
    the other diagonal of its quad, so the links stay a triangulation."""
    rng = np.random.default_rng(22)
    L, K = 48, 14
    for trial in range(8):
        pts = _generic_points(rng, L, K, min_sep=7)
        edges, tris, margin, dual, dual_of = periodic_delaunay(pts, Q * L, Q * L, radius=int(0.8 * L * Q))
        cq = np.array(pts, dtype=np.int64)
        E = O.vertex_edges(O.owners_bruteforce(cq, L, L), cq)
        got = set(zip(*[a_.tolist() for a_ in O.split_keys(E)]))
        assert len(got) == len(edges), trial
        nb = {}
        for x, y in edges:
            nb.setdefault(x, set()).add(y)
            nb.setdefault(y, set()).add(x)
        missed = edges - got
        for e in missed:
            assert dual_of[e] < Q, (trial, e, dual_of[e] / Q)
            # on a small torus two labels can share more than one pair of
            # neighbours (through different images); the quad is then not
            # named by labels alone
            opp = sorted(nb[e[0]] & nb[e[1]])
            if len(opp) == 2:
                assert (opp[0], opp[1]) in got, (trial, e, opp)
        assert len(got - edges) == len(missed), trial


def _links_cross(cq, E, M):
    """Whether two links, drawn as the shortest segments between their centres
    on the M x M torus, cross at a point inside both (shared ends excluded)."""
    i, j = O.split_keys(E)
    seg = []
    for p, q in zip(i.tolist(), j.tolist()):
        d = np.array([O.wrap(int(cq[q, t] - cq[p, t]), M) for t in (0, 1)], dtype=np.int64)
        seg.append((p, q, cq[p].astype(np.int64), d))

    def orient(a, b, c):
        return np.sign((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))

    for u in range(len(seg)):
        p, q, a, da = seg[u]
        for w in range(u + 1, len(seg)):
            r, s_, b, db = seg[w]
            if len({p, q, r, s_}) < 4:
                continue
            b0 = a + np.array([O.wrap(int(b[0] - a[0]), M), O.wrap(int(b[1] - a[1]), M)], dtype=np.int64)
            for sx in (-1, 0, 1):
                for sy in (-1, 0, 1):
                    c0 = b0 + np.array([sx * M, sy * M], dtype=np.int64)
                    if (orient(a, a + da, c0) * orient(a, a + da, c0 + db) < 0
                            and orient(c0, c0 + db, a) * orient(c0, c0 + db, a + da) < 0):
                        return True
    return False


def test_vertex_rule_is_a_triangulation_on_dense_random_sets():
    """Cells as close as 3 sites, many of them slivers: the frame rule's links
    still form a triangulation of the torus -- no two links cross, and there
    are E = 3K of them (Euler). Dropping the inner-frame test adds crossing
    links; dropping the second neighbours loses links."""
    rng = np.random.default_rng(7)
    L, K = 40, 40
    for trial in range(4):
        pts = _generic_points(rng, L, K, min_sep=3)
        cq = np.array(pts, dtype=np.int64)
        E = O.vertex_edges(O.owners_bruteforce(cq, L, L), cq)
        assert len(E) == 3 * len(pts), trial
        assert not _links_cross(cq, E, Q * L), trial


@pytest.mark.parametrize("a,b,M,L", [(1, -1, 4, 8), (1, 1, 4, 8), (1, -1, 8, 16), (1, 1, 8, 16),
                                     (2, 1, 4, 8), (1, 2, 4, 8)])
def test_vertex_rule_keeps_one_site_bands_apart(a, b, M, L):
    """Colour (a x + b y) mod M: M bands one site thin, every site a vertex
    site (eight colour changes around each frame). Band c touches only bands
    c - 1 and c + 1, and the frame rule reads exactly that ring whatever the
    centres: across a diagonal band the short-diagonal condition stops the
    second neighbour (x +- y), and across a steep band the long-diagonal
    condition stops the first neighbour (2x + y, x + 2y)."""
    y, x = np.mgrid[0:L, 0:L]
    own = ((a * x + b * y) % M).astype(np.int32)
    assert int(O.frame_gaps(own).min()) == 8
    ring = sorted(tuple(sorted((c, (c + 1) % M))) for c in range(M))
    rng = np.random.default_rng(M + 3 * a + b)
    for _ in range(3):
        cq = rng.integers(0, Q * L, size=(M, 2)).astype(np.int64)
        got = sorted(zip(*[v.tolist() for v in O.split_keys(O.vertex_edges(own, cq))]))
        assert got == ring


def test_vertex_rule_reads_nothing_at_an_obstacle_site():
    """The three-cell junction with its vertex site (1, 1) made an obstacle:
    the obstacle is never an end of a link, and the links read at the other
    vertex sites are unchanged."""
    own = np.array([[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 2, 2], [2, 2, 2, 2]], dtype=np.int32)
    cq = np.array([[512, 512], [Q * 2 + 512, 512], [Q + 512, Q * 2 + 512]], dtype=np.int64)
    own[1, 1] = O.OBSTACLE
    assert int(O.frame_gaps(own)[1, 1]) >= 3
    E = O.vertex_edges(own, cq)
    a, b = O.split_keys(E)
    assert ((a >= 0) & (a < b) & (b < 3)).all()
    assert E.tolist() == O.make_keys([0, 0, 1], [1, 2, 2]).tolist()


@pytest.mark.parametrize("centres,diagonal", [
    # the cells of 1 and 3 are equidistant from the junction and nearest: the
    # plaquette centre takes colour 1, so 1-2 is linked and 0-3 is not
    (((1, 1), (5.5, 1.5), (1, 6), (5.5, 5.5)), (1, 2)),
    # all four equidistant (a square of centres): colour 0, so 0-3
    (((1.5, 1.5), (5.5, 1.5), (1.5, 5.5), (5.5, 5.5)), (0, 3)),
])
def test_vertex_rule_tie_at_a_four_cell_junction(centres, diagonal):
    """8 x 8 box, walls on both axes, four 4 x 4 cells (0 lower left, 1 lower
    right, 2 upper left, 3 upper right) meeting at the plaquette centred on
    (3.5, 3.5), whose four sites are the only vertex sites. Both diagonals
    pass the pathology conditions there; the one whose end owns the plaquette
    centre -- nearest centre, ties to the smallest label -- is linked."""
    own = np.zeros((8, 8), dtype=np.int32)
    own[:4, 4:] = 1
    own[4:, :4] = 2
    own[4:, 4:] = 3
    gaps = O.frame_gaps(own, (False, False))
    assert sorted(zip(*np.nonzero(gaps >= 3))) == [(3, 3), (3, 4), (4, 3), (4, 4)]
    cq = np.array([[int(x * Q), int(y * Q)] for x, y in centres], dtype=np.int64)
    got = sorted(zip(*[v.tolist() for v in O.split_keys(O.vertex_edges(own, cq, periodic=(False, False)))]))
    assert got == sorted([(0, 1), (0, 2), (1, 3), (2, 3), diagonal])



# ----------------------------------------------------------------------------
# Walls (bounded axes, the paper's channel) and obstacles (MAXLINK sites)
# ----------------------------------------------------------------------------

def bfs_labels_walls(fg: np.ndarray, connectivity: int, periodic) -> np.ndarray:
    """Flood fill in raster order; a step that crosses a bounded axis is not taken."""
    Ly, Lx = fg.shape
    lab = -np.ones((Ly, Lx), dtype=np.int64)
    if connectivity == 4:
        steps = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    else:
        steps = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0)]
    nxt = 0
    for y in range(Ly):
        for x in range(Lx):
            if fg[y, x] and lab[y, x] < 0:
                lab[y, x] = nxt
                dq = deque([(x, y)])
                while dq:
                    cx, cy = dq.popleft()
                    for dx, dy in steps:
                        nx, ny = cx + dx, cy + dy
                        if not periodic[0] and not 0 <= nx < Lx:
                            continue
                        if not periodic[1] and not 0 <= ny < Ly:
                            continue
                        nx, ny = nx % Lx, ny % Ly
                        if fg[ny, nx] and lab[ny, nx] < 0:
                            lab[ny, nx] = nxt
                            dq.append((nx, ny))
                nxt += 1
    return lab


@pytest.mark.parametrize("periodic", [(False, True), (True, False), (False, False)])
@pytest.mark.parametrize("conn", [4, 8])
def test_ccl_with_walls_matches_bfs(periodic, conn):
    rng = np.random.default_rng(31 + conn + 2 * periodic[0] + 4 * periodic[1])
    for trial in range(150):
        Lx = int(rng.integers(1, 12))
        Ly = int(rng.integers(1, 12))
        fg = rng.random((Ly, Lx)) < float(rng.uniform(0.1, 0.9))
        lab, K = O.label_components(fg, conn, periodic)
        ref = bfs_labels_walls(fg, conn, periodic)
        assert np.array_equal(lab, ref), (trial, Lx, Ly)


def test_walls_split_bubbles_and_keep_plain_centres():
    """A bar touching both x walls is two bubbles when x is bounded (one on the
    torus); each centre is the plain mean of its sites (closed form)."""
    fg = np.zeros((4, 10), dtype=bool)
    fg[1, [0, 1, 8, 9]] = True
    lab, K = O.label_components(fg, 4, (True, True))
    assert K == 1
    lab, K = O.label_components(fg, 4, (False, True))
    assert K == 2
    cq = O.centroids_q10(lab, K, (False, True))
    assert cq.tolist() == [[512, Q], [Q * 8 + 512, Q]]


def test_walls_change_owners_links_and_matches():
    """Centres at x = 1 and x = 8 on a 10-wide lattice own the same halves with
    or without walls; three cells side by side are linked across the seam only
    on the torus; the centre match measures plain distances with walls."""
    cq = np.array([[Q * 1, Q], [Q * 8, Q]], dtype=np.int64)
    own_t = O.owners_bruteforce(cq, 10, 3)
    own_w = O.owners_bruteforce(cq, 10, 3, periodic=(False, True))
    assert own_w[0].tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1, 1]
    assert own_t[0].tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1, 1]
    E_t = O.delaunay_edges(own_t, cq)
    E_w = O.delaunay_edges(own_w, cq, (False, True))
    assert E_t.tolist() == E_w.tolist() == O.make_keys([0], [1]).tolist()
    # three cells side by side: 2 and 0 meet only across the seam
    own = np.zeros((3, 10), dtype=np.int32)
    own[:, 3:7] = 1
    own[:, 7:] = 2
    cq3 = np.array([[Q, Q], [Q * 5, Q], [Q * 8, Q]], dtype=np.int64)
    assert O.delaunay_edges(own, cq3).tolist() == O.make_keys([0, 0, 1], [1, 2, 2]).tolist()
    assert O.delaunay_edges(own, cq3, (False, True)).tolist() == O.make_keys([0, 1], [1, 2]).tolist()
    # centre match: 9.5 sites apart plainly, 0.5 through the seam
    p = np.array([[Q // 4, Q]], dtype=np.int64)
    n = np.array([[Q * 9 + 3 * Q // 4, Q]], dtype=np.int64)
    assert O.match_centroid(p, n, 10, 3, radius=1)[0].tolist() == [0]
    assert O.match_centroid(p, n, 10, 3, radius=1, periodic=(False, True))[0].tolist() == [-1]


def test_obstacles_are_never_bubbles_owners_or_links():
    """An obstacle column splits a bar; its sites get the MAXLINK owner and no
    link touches it, so the two cells beside it are linked only where they
    meet without the obstacle in between."""
    L = 12
    F = np.zeros((L, L), dtype=np.float32)
    F[5, :] = 1.0
    obst = np.zeros((L, L), dtype=bool)
    obst[:, 6] = True
    d = O.Detector(L, L, voronoi="brute", obstacles=obst)
    r = d.push(F)
    assert r["K"] == 1                       # the bar still joins around the seam
    assert (r["labels"][:, 6] == -1).all()
    assert (r["owners"][:, 6] == O.OBSTACLE).all()
    d2 = O.Detector(L, L, voronoi="brute", obstacles=obst, walls=(True, False))
    r2 = d2.push(F)
    assert r2["K"] == 2                      # walls in x and the obstacle: two bars
    for res in (r, r2):
        a, b = O.split_keys(res["edges"])
        assert ((a >= 0) & (a < b) & (b < res["K"])).all()
    assert (r2["owners"][:, 6] == O.OBSTACLE).all()


def test_obstacle_corner_breaks_adjacency_and_plaquette():
    """4 x 4 box with walls on both axes, cells 0 (top left), 1 (top right), 2
    (bottom left), 3 (bottom right) and an obstacle at (2, 2): the plaquette at
    (1, 1) carries 0, 1, the obstacle and 2 -- four distinct values, but not
    four labels, so it gives no diagonal -- and no pair touching the obstacle
    is linked. What remains are the four side adjacencies."""
    X = O.OBSTACLE
    own = np.array([[0, 0, 1, 1],
                    [0, 0, 1, 1],
                    [2, 2, X, 3],
                    [2, 2, 3, 3]], dtype=np.int32)
    cq = np.array([[Q // 2, Q // 2], [Q * 5 // 2, Q // 2], [Q // 2, Q * 5 // 2], [Q * 5 // 2, Q * 5 // 2]],
                  dtype=np.int64)
    E = O.delaunay_edges(own, cq, (False, False))
    assert E.tolist() == O.make_keys([0, 0, 1, 2], [1, 2, 3, 3]).tolist()


@pytest.mark.parametrize("periodic", [(False, True), (True, False), (False, False)])
def test_owners_with_walls_equal_plain_loops(periodic):
    """Owners on bounded axes: nearest centre by plain (not wrapped) squared
    distance along a bounded axis, ties to the smallest label, checked by a
    pure-Python double loop."""
    rng = np.random.default_rng(91 + 2 * periodic[0] + periodic[1])
    Lx, Ly = 13, 9
    cq = rng.integers(0, [Q * Lx, Q * Ly], size=(6, 2))
    cq[5] = cq[2]                     # an exact tie: label 2 must win
    own = O.owners_bruteforce(cq, Lx, Ly, periodic=periodic)
    for y in range(Ly):
        for x in range(Lx):
            best, bi = None, -1
            for i, (cx, cy) in enumerate(cq.tolist()):
                dx = Q * x - cx
                dy = Q * y - cy
                if periodic[0]:
                    dx = (dx + Q * Lx // 2) % (Q * Lx) - Q * Lx // 2
                if periodic[1]:
                    dy = (dy + Q * Ly // 2) % (Q * Ly) - Q * Ly // 2
                d = dx * dx + dy * dy
                if best is None or d < best:
                    best, bi = d, i
            assert own[y, x] == bi, (x, y)


def test_frame_is_truncated_at_a_wall():
    """A site on the x = 0 wall keeps five frame neighbours (+x, +x+y, +y, -y,
    +x-y in cyclic order); their colours 1,1,1,0,0 change twice around the
    frame, so it is not a vertex with walls, while on the torus the three
    neighbours beyond the seam (colour 2) make a third change."""
    own = np.zeros((5, 6), dtype=np.int32)
    own[:, 5] = 2                     # the column beyond the seam on the torus
    own[2, 1] = 1                     # +x of the site (0, 2)
    own[3, 1] = 1                     # +x+y
    own[3, 0] = 1                     # +y
    g_wall = O.frame_gaps(own, (False, True))
    g_torus = O.frame_gaps(own)
    assert int(g_wall[2, 0]) == 2
    assert int(g_torus[2, 0]) >= 3


# ----------------------------------------------------------------------------
# Symmetries that any correct reading of the match and the flips must have
# ----------------------------------------------------------------------------

def test_matches_are_symmetric_in_time():
    """Mutual best overlap and mutual nearest centres do not depend on which
    frame is called past: swapping the frames swaps Phi and its inverse."""
    rng = np.random.default_rng(5)
    for trial in range(8):
        L = int(rng.integers(24, 64))
        F0 = I.smoothed_noise(L, L, 2.5, seed=trial)
        F1 = I.shear_resample(F0, 0.05, 0.05, np.random.default_rng(trial))
        l0, k0 = O.label_components(O.foreground(F0))
        l1, k1 = O.label_components(O.foreground(F1))
        phi, inv = O.match_overlap(l0, l1, k0, k1)
        phi_r, inv_r = O.match_overlap(l1, l0, k1, k0)
        assert phi.tolist() == inv_r.tolist() and inv.tolist() == phi_r.tolist()
        c0, c1 = O.centroids_q10(l0, k0), O.centroids_q10(l1, k1)
        phi, inv = O.match_centroid(c0, c1, L, L, radius=5)
        phi_r, inv_r = O.match_centroid(c1, c0, L, L, radius=5)
        assert phi.tolist() == inv_r.tolist() and inv.tolist() == phi_r.tolist()


def test_flips_reverse_in_time():
    """Run backwards, a breaking link becomes an arising one: the arising links
    from past to now, written in past labels, are the breaking links from now
    to past, and the other way round."""
    rng = np.random.default_rng(6)
    checked = 0
    for trial in range(10):
        L = int(rng.integers(40, 80))
        F0 = I.smoothed_noise(L, L, 3.0, seed=20 + trial)
        F1 = I.shear_resample(F0, 0.08, 0.05, np.random.default_rng(trial))
        d = O.Detector(L, L, voronoi="brute")
        a = d.push(F0)
        b = d.push(F1)
        phi, inv = b["phi"], b["inv"]
        fwd = O.flips(a["edges"], b["edges"], phi, inv)
        bwd = O.flips(b["edges"], a["edges"], inv, phi)
        # arising (now labels) -> past labels, against breaking of the reversed run
        x, y = O.split_keys(fwd["arising"])
        arising_in_past = np.sort(O.make_keys(inv[x], inv[y])) if x.size else np.zeros(0, np.uint64)
        assert arising_in_past.tolist() == bwd["breaking"].tolist()
        x, y = O.split_keys(bwd["arising"])
        back = np.sort(O.make_keys(phi[x], phi[y])) if x.size else np.zeros(0, np.uint64)
        assert back.tolist() == fwd["breaking"].tolist()
        checked += int(fwd["breaking"].size + fwd["arising"].size > 0)
    assert checked >= 3


def test_event_classes_reverse_in_time():
    """The event classes use both triangulations alike: run backwards, every
    active label keeps its bulk and boundary event classes, and its boundary
    point flags of the past and the now triangulation trade places."""
    rng = np.random.default_rng(8)
    seen = 0
    for trial in range(16):
        L = int(rng.integers(48, 96))
        F0 = I.smoothed_noise(L, L, float(rng.uniform(2.0, 4.0)), seed=40 + trial)
        F1 = I.shear_resample(F0, 0.2, 0.05, np.random.default_rng(trial))
        d = O.Detector(L, L, voronoi="brute")
        a = d.push(F0)
        b = d.push(F1)
        phi, inv = b["phi"], b["inv"]
        fwd = O.flips(a["edges"], b["edges"], phi, inv)
        bwd = O.flips(b["edges"], a["edges"], inv, phi)
        ef = O.classify_events(a["edges"], b["edges"], phi, inv, fwd["active"])
        eb = O.classify_events(b["edges"], a["edges"], inv, phi, bwd["active"])
        for n in np.flatnonzero(ef).tolist():
            p = int(inv[n])
            f, g = int(ef[n]), int(eb[p])
            assert (f & (O.EV_ACTIVE | O.EV_BULK | O.EV_BOUNDARY)) == (g & (O.EV_ACTIVE | O.EV_BULK | O.EV_BOUNDARY))
            assert bool(f & O.EV_BPOINT_NOW) == bool(g & O.EV_BPOINT_PAST)
            assert bool(f & O.EV_BPOINT_PAST) == bool(g & O.EV_BPOINT_NOW)
            seen += 1
        assert int((eb != 0).sum()) == int((ef != 0).sum())
    assert seen > 20
