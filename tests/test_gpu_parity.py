"""GPU parity: libvd (through its C ABI) against the CPU oracle, bit for bit.

Every output is integer, so the tolerance is exact (0) for labels, Q10
centroids, Voronoi owners, sorted link keys, the isomorphism Phi and the
breaking/arising lists. Sizes span several 64x32 labelling tiles and 32x32
Voronoi tiles with ragged tails; full-size workloads check every output the
oracle can produce in seconds and sampled Voronoi owners (brute force per
site) where the full oracle is slower.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402

FULL = os.environ.get("VD_FULL", "0") == "1"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    vd.lib()


def check_frame(det, r, what=("labels", "centroids", "owners", "edges", "changes"), tag=""):
    K, E, _ = det.counts()
    assert K == r["K"], (tag, "K", K, r["K"])
    if "labels" in what:
        got = det.labels()
        if not np.array_equal(got, r["labels"]):
            bad = np.argwhere(got != r["labels"])
            raise AssertionError(f"{tag} labels differ at {len(bad)} sites, first {bad[:5].tolist()}")
    if "centroids" in what:
        got = det.centroids()
        if not np.array_equal(got, r["centroids"]):
            bad = np.flatnonzero((got != r["centroids"]).any(axis=1))
            raise AssertionError(f"{tag} centroids differ for {len(bad)} bubbles: {bad[:5].tolist()} "
                                 f"got {got[bad[:3]].tolist()} want {r['centroids'][bad[:3]].tolist()}")
    if "owners" in what:
        got = det.owners()
        if not np.array_equal(got, r["owners"]):
            bad = np.argwhere(got != r["owners"])
            raise AssertionError(f"{tag} owners differ at {len(bad)} sites, first {bad[:5].tolist()}")
    if "edges" in what:
        got = det.edges()
        assert E == len(r["edges"]), (tag, "E", E, len(r["edges"]))
        assert np.array_equal(got, r["edges"]), f"{tag} edge keys differ"
    if "changes" in what:
        ch = det.changes()
        assert ch["K_prev"] == r["K_prev"], (tag, ch["K_prev"], r["K_prev"])
        assert ch["n_matched"] == r["n_matched"], (tag, "matched", ch["n_matched"], r["n_matched"])
        assert np.array_equal(ch["breaking"], r["breaking"]), f"{tag} breaking differs"
        assert np.array_equal(ch["breaking_prev"], r["breaking_prev"]), f"{tag} breaking_prev differs"
        assert np.array_equal(ch["arising"], r["arising"]), f"{tag} arising differs"
        assert np.array_equal(ch["active"], r["active"]), f"{tag} active differs"
        assert ch["global_trigger"] == r["global_trigger"]
        if r["K_prev"]:
            assert np.array_equal(det.match(), r["phi"]), f"{tag} phi differs"


def run_pair(frames, threshold=0.5, polarity=1, voronoi="kdtree", what=None, tag="", events=False,
             match="overlap", match_radius=0, connectivity=4, edge_rule="adj4", walls=(False, False),
             obstacles=None):
    Ly, Lx = frames[0].shape
    det = vd.Detector(Lx, Ly, threshold=threshold, polarity=polarity, events=events,
                      match_rule=vd.VD_MATCH_CENTROID if match == "centroid" else vd.VD_MATCH_OVERLAP,
                      match_radius=match_radius, connectivity=connectivity,
                      edge_rule=vd.VD_EDGE_VERTEX if edge_rule == "vertex" else vd.VD_EDGE_ADJ4,
                      walls=(vd.VD_WALL_X if walls[0] else 0) | (vd.VD_WALL_Y if walls[1] else 0))
    if obstacles is not None:
        det.set_obstacles(obstacles)
    ref = O.Detector(Lx, Ly, theta=threshold, polarity=polarity, voronoi=voronoi, workers=-1, events=events,
                     match=match, match_radius=match_radius, connectivity=connectivity, edge_rule=edge_rule,
                     walls=walls, obstacles=obstacles)
    for f, F in enumerate(frames):
        det.push(torch.from_numpy(np.ascontiguousarray(F)).cuda())
        r = ref.push(F)
        check_frame(det, r, tag=f"{tag} frame {f}", **({} if what is None else {"what": what}))
    det.close()
    return r


def test_c0_two_frames():
    r = run_pair(I.workload_c0(seed=1), tag="c0")
    assert r["K"] > 10


@pytest.mark.parametrize("seed", range(6))
def test_random_small_lattices(seed):
    """Random sizes (1..150, ragged against both tilings), densities and polarity."""
    rng = np.random.default_rng(100 + seed)
    for trial in range(6):
        Lx = int(rng.integers(1, 150))
        Ly = int(rng.integers(1, 150))
        if trial % 3 == 0:
            F0 = rng.random((Ly, Lx)).astype(np.float32)
            F1 = np.where(rng.random((Ly, Lx)) < 0.1, rng.random((Ly, Lx)), F0).astype(np.float32)
            thr = float(rng.uniform(0.2, 0.8))
        else:
            sig = float(rng.uniform(1.0, 4.0))
            F0 = I.smoothed_noise(Ly, Lx, sig, seed=seed * 10 + trial)
            F1 = I.shear_resample(F0, 0.03, 0.02, np.random.default_rng(trial))
            thr = float(rng.uniform(-0.5, 1.0))
        pol = 1 if rng.random() < 0.7 else -1
        run_pair([F0, F1], threshold=thr, polarity=pol, voronoi="brute", tag=f"{Lx}x{Ly} pol{pol}")


def test_degenerate_fields():
    L = 70
    cases = {
        "empty": np.zeros((L, L), np.float32),
        "full": np.ones((L, L), np.float32),
        "checker": ((np.indices((L, L)).sum(0) % 2) == 0).astype(np.float32),
        "stripes": np.tile((np.arange(L) % 3 == 0).astype(np.float32), (L, 1)),
        "single": np.pad(np.ones((1, 1), np.float32), ((5, L - 6), (9, L - 10))),
        "nan": np.where(np.random.default_rng(0).random((L, L)) < 0.3, np.nan, 1.0).astype(np.float32),
    }
    for name, F in cases.items():
        run_pair([F, np.roll(F, 1, axis=1)], voronoi="brute", tag=name)


@pytest.mark.parametrize("connectivity", [4, 8])
def test_pieces_per_tile_at_the_shared_sum_limit(connectivity):
    """Labelling tiles (64 x 32 sites) holding 31, 32, 33, 1, 0, 200, 64 and 65
    pieces: a tile of up to 32 pieces sums them in shared memory, a larger one
    with global atomics, and both must give the oracle's labels, sizes and
    centres. Pieces are two-site runs three columns and two rows apart; the
    second frame shifts them by three columns, so the last column of pieces
    crosses the tile seams (and the lattice's periodic edge)."""
    L = 128
    F = np.zeros((L, L), np.float32)
    counts = [31, 32, 33, 1, 0, 200, 64, 65]
    slots = [(3 * a, 2 * b) for b in range(16) for a in range(21)]
    for t, n in enumerate(counts):
        x0, y0 = 64 * (t % 2), 32 * (t // 2)
        for (x, y) in slots[:n]:
            F[y0 + y, x0 + x:x0 + x + 2] = 1.0
    r = run_pair([F, np.roll(F, 3, axis=1)], voronoi="brute", connectivity=connectivity, tag=f"pcap c{connectivity}")
    assert r["K"] == sum(counts)


def test_wide_bubbles_across_seams():
    """Bubbles wider than half the lattice and winding ones take the exact path."""
    for L in (40, 64, 96, 130):
        F = np.zeros((L, L), np.float32)
        F[3, :] = 1.0                              # winds around x
        F[:, 7] = 1.0                              # winds around y (joined with the row)
        F[10:14, 2: L - 5] = 1.0                   # wider than L/2
        F[L - 3:, L - 3:] = 1.0                    # corner block across both seams
        F[:2, :2] = 1.0
        F[20: 20 + L // 2 + 3, 30 % L] = 1.0       # tall bar
        run_pair([F, np.roll(F, 2, axis=0)], voronoi="brute", tag=f"wide{L}")


def test_tiny_lattices():
    rng = np.random.default_rng(5)
    for Lx, Ly in [(1, 1), (1, 7), (7, 1), (2, 2), (3, 2), (1, 64), (64, 1), (65, 33), (33, 65)]:
        F0 = rng.random((Ly, Lx)).astype(np.float32)
        F1 = rng.random((Ly, Lx)).astype(np.float32)
        run_pair([F0, F1], voronoi="brute", tag=f"tiny{Lx}x{Ly}")


def test_pitched_field():
    F = I.smoothed_noise(100, 90, 2.5, seed=3)
    big = np.zeros((100, 96), np.float32)
    big[:, :90] = F
    det = vd.Detector(90, 100)
    t = torch.from_numpy(big).cuda()[:, :90]
    det.push(t)
    r = O.Detector(90, 100).push(F)
    check_frame(det, r, what=("labels", "centroids", "owners", "edges"), tag="pitched")


def test_host_push_matches_device_push():
    frames = I.workload_c0(seed=4)
    a = vd.Detector(128, 128)
    b = vd.Detector(128, 128)
    for F in frames:
        a.push(torch.from_numpy(F).cuda())
        b.push_host(F)
        assert np.array_equal(a.labels(), b.labels())
        assert np.array_equal(a.edges(), b.edges())
        ca, cb = a.changes(), b.changes()
        assert np.array_equal(ca["breaking"], cb["breaking"]) and np.array_equal(ca["arising"], cb["arising"])


def test_c1_frames():
    """1024x1024 smoothed noise (sigma 4), sheared frame to frame: full oracle each frame."""
    n = 64
    frames = list(I.workload_c1(seed=1, n_frames=n))
    r = run_pair(frames, tag="c1")
    assert r["K"] > 500


def test_c2_frames():
    """4096x4096 RSA droplets: labels, centroids, links and flips from the full oracle."""
    n = 16
    frames = [F for F, _ in I.workload_c2(seed=1, n_frames=n)]
    r = run_pair(frames, tag="c2")
    assert r["K"] > 20000


def test_c2_sampled_owners_bruteforce():
    """Voronoi owners at full size, sampled sites checked by the all-centres definition."""
    F, st = next(iter(I.workload_c2(seed=2, n_frames=1)))
    L = F.shape[0]
    det = vd.Detector(L, L)
    det.push(torch.from_numpy(F).cuda())
    lab, K = O.label_components(O.foreground(F))
    cq = O.centroids_q10(lab, K)
    assert np.array_equal(det.centroids(), cq)
    own = det.owners().ravel()
    rng = np.random.default_rng(0)
    sites = rng.choice(L * L, size=4000, replace=False)
    want = O.owners_bruteforce(cq, L, L, sites=sites)
    assert np.array_equal(own[sites], want)


def test_capacity_overflow_is_reported():
    F = ((np.indices((64, 64)).sum(0) % 2) == 0).astype(np.float32)   # 2048 bubbles
    det = vd.Detector(64, 64, max_components=100)
    det.push(torch.from_numpy(F).cuda())
    with pytest.raises(vd.VdError) as e:
        det.labels()
    assert e.value.status == vd.VD_ERR_CAPACITY
    # the context stays usable after a capacity error on a fitting frame
    G = np.zeros((64, 64), np.float32)
    G[10:20, 10:20] = 1.0
    det.push(torch.from_numpy(G).cuda())
    assert det.counts()[0] == 1


def test_link_capacity_overflow_then_exact_frames():
    """A frame with more links than max_edges reports VD_ERR_CAPACITY; the
    frames after it (with fewer links) are exact in every output: no count
    of the overflowed frame carries over into their adjacency."""
    L = 128
    dense = I.smoothed_noise(L, L, 1.5, seed=3)
    sparse = list(I.noise_frames(L, 5.0, 2, 0.02, seed=4))
    ref = O.Detector(L, L, voronoi="brute")
    r_dense = ref.push(dense)
    few = [ref.push(F) for F in sparse]
    cap = max(len(r["edges"]) for r in few) + 8
    assert len(r_dense["edges"]) > cap, "the dense frame must overflow the link capacity"
    det = vd.Detector(L, L, max_edges=cap)
    det.push(torch.from_numpy(dense).cuda())
    with pytest.raises(vd.VdError) as e:
        det.edges()
    assert e.value.status == vd.VD_ERR_CAPACITY
    for f, (F, r) in enumerate(zip(sparse, few)):
        det.push(torch.from_numpy(F).cuda())
        what = ("labels", "centroids", "owners", "edges") if f == 0 else ("labels", "centroids", "owners", "edges", "changes")
        check_frame(det, r, what=what, tag=f"after overflow, frame {f}")
    det.close()


def test_overlap_capacity_overflow_then_exact_frames():
    """20 horizontal stripes followed by 20 vertical ones overlap in 400
    (past, now) pairs, more than the overlap list of a context capped at 100
    bubbles holds (2 * 100 + 64): that frame reports VD_ERR_CAPACITY, and the
    frames after it are exact again."""
    L = 80
    horiz = np.zeros((L, L), np.float32)
    horiz[(np.arange(L) % 4) < 2, :] = 1.0
    vert = np.ascontiguousarray(horiz.T)
    blobs = list(I.noise_frames(L, 3.0, 2, 0.02, seed=8))
    frames = [horiz, vert] + blobs
    ref = O.Detector(L, L, voronoi="brute")
    want = [ref.push(F) for F in frames]
    det = vd.Detector(L, L, max_components=100)
    for f, (F, r) in enumerate(zip(frames, want)):
        det.push(torch.from_numpy(F).cuda())
        if f == 1:
            with pytest.raises(vd.VdError) as e:
                det.changes()
            assert e.value.status == vd.VD_ERR_CAPACITY
            continue
        what = ("labels", "centroids", "owners", "edges") if f == 2 else ("labels", "centroids", "owners", "edges",
                                                                          "changes")
        check_frame(det, r, what=what, tag=f"frame {f}")
    det.close()


def test_piece_pool_overflow_then_exact_frames():
    """A 512^2 checkerboard has 131,072 one-site bubbles: more tile pieces
    than the step's piece pool holds (N / 8 + 16 per tile above 65,536 sites)
    and more bubbles than the default capacity. The frame reports
    VD_ERR_CAPACITY; the frames after it are exact in every output."""
    L = 512
    checker = ((np.indices((L, L)).sum(0) % 2) == 0).astype(np.float32)
    frames = list(I.noise_frames(L, 4.0, 2, 0.01, seed=12))
    ref = O.Detector(L, L)
    want = [ref.push(F) for F in frames]
    det = vd.Detector(L, L)
    det.push(torch.from_numpy(checker).cuda())
    with pytest.raises(vd.VdError) as e:
        det.labels()
    assert e.value.status == vd.VD_ERR_CAPACITY
    for f, (F, r) in enumerate(zip(frames, want)):
        det.push(torch.from_numpy(F).cuda())
        what = ("labels", "centroids", "owners", "edges") if f == 0 else ("labels", "centroids", "owners", "edges",
                                                                          "changes")
        check_frame(det, r, what=what, tag=f"after overflow, frame {f}")
    det.close()


def test_event_classes_with_boundary_points():
    """Few large bubbles (64 x 64, sigma 6): the digital link graph of frame 1
    is not a full triangulation of the torus, so some active labels are
    boundary points (a link whose ends share one neighbour) and boundary event
    points (Section 3.2.4). The flags must equal the oracle's; the oracle is
    checked to show the boundary class, so the case keeps its point."""
    frames = list(I.noise_frames(64, 6.0, 5, 0.05, 18))
    ref = O.Detector(64, 64, events=True)
    rs = [ref.push(F) for F in frames]
    assert any(int((r["active"] & O.EV_BOUNDARY).sum()) for r in rs)
    run_pair(frames, tag="events 64", events=True)


@pytest.mark.parametrize("radius", [1, 3, 12])
def test_centroid_match_sequences(radius):
    """Isomorphism by centres (VD_MATCH_CENTROID): sheared smoothed noise on a
    lattice ragged against the tiles, with the event classes on. Phi, the flips
    and the flags must equal the oracle's; radius 1 leaves many labels
    unmatched, 12 reaches across several buckets."""
    F = I.smoothed_noise(136, 200, 3.0, seed=radius)
    frames = [F]
    for k in range(3):
        frames.append(I.shear_resample(frames[-1], 0.02, 0.01, np.random.default_rng(k + 10 * radius)))
    r = run_pair(frames, tag=f"centroid r{radius}", events=True, match="centroid", match_radius=radius)
    assert r["K"] > 10


def test_centroid_match_c1_frames():
    """1024x1024 smoothed noise, centre match within 8 sites, event classes on."""
    frames = list(I.workload_c1(seed=2, n_frames=3))
    r = run_pair(frames, tag="c1 centroid", events=True, match="centroid", match_radius=8)
    assert r["n_matched"] > 0.8 * r["K"]


def test_centroid_match_in_batches():
    """Sequence and independent batches with the centre match: every frame's
    changes equal the oracle run frame by frame (the past grid of a sequence
    instance is the previous instance's grid of the same push)."""
    frames = list(I.noise_frames(256, 3.0, 6, 0.01, 5))
    dev = [torch.from_numpy(np.ascontiguousarray(F)).cuda() for F in frames]
    ref = O.Detector(256, 256, events=True, match="centroid", match_radius=6)
    rs = [ref.push(F) for F in frames]
    seq = vd.Batch([(256, 256)], sequence=3, events=True, match_rule=vd.VD_MATCH_CENTROID, match_radius=6)
    for p in range(2):
        seq.push(dev[3 * p:3 * p + 3])
        for i in range(3):
            r = rs[3 * p + i]
            ch = seq.changes(i)
            assert np.array_equal(ch["breaking"], r["breaking"]), (p, i)
            assert np.array_equal(ch["arising"], r["arising"]), (p, i)
            assert np.array_equal(ch["active"], r["active"]), (p, i)
    seq.close()


@pytest.mark.parametrize("seed", range(4))
def test_eight_connectivity(seed):
    """8-connected bubbles (Section 3.1 with the diagonal lattice directions):
    random fields on lattices ragged against the 64 x 32 tiles, including
    one-tile-wide and one-row tori, and smoothed noise across tile corners."""
    rng = np.random.default_rng(300 + seed)
    for trial in range(5):
        Lx = int(rng.integers(1, 200))
        Ly = int(rng.integers(1, 120))
        if trial % 2 == 0:
            p = float(rng.uniform(0.2, 0.6))
            F0 = (rng.random((Ly, Lx)) < p).astype(np.float32)
            F1 = np.where(rng.random((Ly, Lx)) < 0.05, 1.0 - F0, F0).astype(np.float32)
        else:
            F0 = I.smoothed_noise(Ly, Lx, float(rng.uniform(1.0, 3.0)), seed=seed * 10 + trial)
            F1 = I.shear_resample(F0, 0.03, 0.02, np.random.default_rng(trial))
        run_pair([F0, F1], voronoi="brute", tag=f"c8 {Lx}x{Ly}", connectivity=8)


def test_eight_connectivity_c1_frames():
    """1024x1024 smoothed noise with 8-connected bubbles: full oracle."""
    frames = list(I.workload_c1(seed=3, n_frames=3))
    r = run_pair(frames, tag="c1 c8", connectivity=8)
    assert r["K"] > 300


@pytest.mark.parametrize("seed", range(3))
def test_vertex_link_rule(seed):
    """The paper's vertex / frame link rule (VD_EDGE_VERTEX): links, Phi, flips
    and event flags equal the oracle's reading of it, on lattices ragged against
    the 32 x 32 link tiles, with bubbles from a handful to a few hundred."""
    rng = np.random.default_rng(500 + seed)
    for trial in range(3):
        Lx = int(rng.integers(16, 260))
        Ly = int(rng.integers(16, 200))
        sig = float(rng.uniform(1.5, 4.0))
        F0 = I.smoothed_noise(Ly, Lx, sig, seed=seed * 10 + trial)
        F1 = I.shear_resample(F0, 0.03, 0.02, np.random.default_rng(trial))
        run_pair([F0, F1], voronoi="brute", tag=f"vertex {Lx}x{Ly}", edge_rule="vertex", events=True)


@pytest.mark.parametrize("L,sigma,seed", [(256, 1.0, 0), (128, 1.0, 2), (200, 1.3, 4)])
def test_vertex_link_rule_inner_frame_colour(L, sigma, seed):
    """Dense small bubbles, where the Voronoi colour of a plaquette centre is
    sometimes a centre that owns none of the plaquette's corner sites (on
    these seeded frames that decides between 8 and 33 diagonals): the
    vertex rule's links equal the oracle's, which colours the inner-frame
    point by the exact nearest centre over all centres."""
    frames = list(I.noise_frames(L, sigma, 2, 0.03, seed=seed))
    run_pair(frames, tag=f"vertex dense {L} {sigma}", edge_rule="vertex", events=True)


def test_vertex_link_rule_c1_frames():
    """1024x1024 smoothed noise with the vertex rule: full oracle."""
    frames = list(I.workload_c1(seed=4, n_frames=3))
    r = run_pair(frames, tag="c1 vertex", edge_rule="vertex")
    assert r["K"] > 300


@pytest.mark.parametrize("walls", [(True, False), (False, True), (True, True)])
def test_walls_and_obstacles(walls):
    """Bounded axes (the paper's channel) with posts along one wall: labels,
    centres, owners (obstacles = VD_OWNER_OBSTACLE), links of both rules,
    the centre match and the event flags equal the oracle's, on lattices
    ragged against the tiles."""
    rng = np.random.default_rng(700 + walls[0] + 2 * walls[1])
    for trial in range(3):
        Lx = int(rng.integers(20, 200))
        Ly = int(rng.integers(20, 150))
        F0 = I.smoothed_noise(Ly, Lx, float(rng.uniform(1.5, 3.5)), seed=trial + 7)
        F1 = I.shear_resample(F0, 0.03, 0.02, np.random.default_rng(trial))
        obst = np.zeros((Ly, Lx), dtype=bool)
        for y0 in range(2, Ly - 4, 12):          # posts on the left wall
            obst[y0:y0 + 4, 0:3] = True
        if trial == 1:
            obst |= rng.random((Ly, Lx)) < 0.01  # and scattered obstacle sites
        tag = f"walls {walls} {Lx}x{Ly} t{trial}"
        run_pair([F0, F1], voronoi="brute", tag=tag, walls=walls, obstacles=obst if trial else None, events=True)
        run_pair([F0, F1], voronoi="brute", tag=tag + " vertex", walls=walls, obstacles=obst, edge_rule="vertex",
                 match="centroid", match_radius=6, events=True)
